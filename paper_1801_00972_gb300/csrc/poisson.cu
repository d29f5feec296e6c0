// Geometric multigrid solve of the discrete Poisson equation (Eq. 3)
//     (sum of the 6 neighbours - 6 phi) / dx^2 = -rho / eps0
// on the cell-corner nodes, periodic in x and y, Dirichlet electrode planes
// k = 0 and k = nz.  The paper factorises the same matrix once with SuperLU
// and back-solves each step; here the solution comes from iterative
// refinement in FP64:
//     r = f - A phi            (FP64, fused with the previous correction)
//     A e = r                  (one V(2,2) cycle in T = float or double)
//     phi += e
// until ||r|| <= tol ||b||, b = f plus the electrode terms.  A V-cycle uses
// red-black Gauss-Seidel smoothing, full-weighting restriction, trilinear
// prolongation, the 7-point operator rediscretised on each level (spacing
// doubling), and many smoothing sweeps on the coarsest level in one block.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "pic_internal.cuh"

#ifndef PIC_MG_PRE
#define PIC_MG_PRE 2
#endif
#ifndef PIC_MG_POST
#define PIC_MG_POST 2
#endif
#ifndef PIC_MG_OMEGA
#define PIC_MG_OMEGA 1.0
#endif

namespace pic {
namespace {

constexpr int kPre = PIC_MG_PRE;         // pre-smoothing sweeps of a V-cycle
constexpr int kPost = PIC_MG_POST;       // post-smoothing sweeps
constexpr double kOmega = PIC_MG_OMEGA;  // relaxation factor of the red-black Gauss-Seidel sweeps

struct Dims {
    int nx, ny, nz;
};

__device__ __forceinline__ size_t nid(const Dims& d, int i, int j, int k)
{
    return ((size_t)k * d.ny + j) * d.nx + i;
}

// The stencil kernels run on 3-D grids: threads over (i, j) of a plane, one
// grid row of blocks per k; all indices are 32-bit (a mesh has < 2^31 nodes).
struct Grid3 {
    dim3 grid, block;
};
inline Grid3 grid3(int nx, int ny, int planes)
{
    const int bx = nx >= 32 ? 32 : nx;
    const int by = std::max(1, std::min(ny, 256 / bx));
    return Grid3{dim3((unsigned)((nx + bx - 1) / bx), (unsigned)((ny + by - 1) / by), (unsigned)planes),
                 dim3((unsigned)bx, (unsigned)by, 1)};
}

__device__ __forceinline__ int tid_flat() { return threadIdx.y * blockDim.x + threadIdx.x; }

// red-black Gauss-Seidel, one colour; thread (i2, j) of plane k = 1 + blockIdx.z
template <typename T>
__global__ void k_rbgs(T* __restrict__ u, const T* __restrict__ f, Dims d, T h2, int color, int zero)
{
    const int i2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = 1 + blockIdx.z;
    if (i2 >= d.nx / 2 || j >= d.ny) return;
    const int i = 2 * i2 + ((j + k + color) & 1);
    const int P = d.nx * d.ny;
    const int n = k * P + j * d.nx + i;
    if (zero) {   // first sweep from a zero guess: the neighbours are still zero
        u[n] = (T)kOmega * (h2 * f[n]) * (T)(1.0 / 6.0);
        return;
    }
    const int row = n - i;
    const int ip = (i + 1 == d.nx) ? 0 : i + 1, im = (i == 0) ? d.nx - 1 : i - 1;
    const int jp = (j + 1 == d.ny) ? -j * d.nx : d.nx, jm = (j == 0) ? (d.ny - 1) * d.nx : -d.nx;
    const T s = u[row + ip] + u[row + im] + u[n + jp] + u[n + jm] + u[n + P] + u[n - P];
    const T gs = (s + h2 * f[n]) * (T)(1.0 / 6.0);
    u[n] = kOmega == 1.0 ? gs : u[n] + (T)kOmega * (gs - u[n]);
}

// r = f - A u on the interior planes (the electrode planes of r stay zero)
template <typename T>
__global__ void k_resid(const T* __restrict__ u, const T* __restrict__ f, T* __restrict__ r, Dims d, T inv_h2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = 1 + blockIdx.z;
    if (i >= d.nx || j >= d.ny) return;
    const int P = d.nx * d.ny;
    const int n = k * P + j * d.nx + i;
    const int row = n - i;
    const int ip = (i + 1 == d.nx) ? 0 : i + 1, im = (i == 0) ? d.nx - 1 : i - 1;
    const int jp = (j + 1 == d.ny) ? -j * d.nx : d.nx, jm = (j == 0) ? (d.ny - 1) * d.nx : -d.nx;
    const T s = u[row + ip] + u[row + im] + u[n + jp] + u[n + jm] + u[n + P] + u[n - P];
    r[n] = f[n] - ((T)6 * u[n] - s) * inv_h2;
}

// full weighting: weights (1/4, 1/2, 1/4) per axis around the coincident fine
// node; thread (I, J) of coarse plane K = 1 + blockIdx.z
template <typename T>
__global__ void k_restrict(const T* __restrict__ rf, T* __restrict__ fc, Dims df, Dims dc)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = 1 + blockIdx.z;
    if (I >= dc.nx || J >= dc.ny) return;
    const int Pf = df.nx * df.ny;
    const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * K;
    const int im = (i0 == 0) ? df.nx - 1 : i0 - 1, ip = i0 + 1;   // i0 + 1 < nx (nx even)
    const int jm = (j0 == 0) ? df.ny - 1 : j0 - 1, jp = j0 + 1;
    const int cols[3] = {im, i0, ip};
    const int rows[3] = {jm * df.nx, j0 * df.nx, jp * df.nx};
    const T w[3] = {(T)0.25, (T)0.5, (T)0.25};
    T acc = (T)0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int pl = (k0 - 1 + a) * Pf;
        T pa = (T)0;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const T* rr = rf + pl + rows[b];
            pa += w[b] * (w[0] * rr[cols[0]] + w[1] * rr[cols[1]] + w[2] * rr[cols[2]]);
        }
        acc += w[a] * pa;
    }
    fc[K * dc.nx * dc.ny + J * dc.nx + I] = acc;
}

// restriction of the residual f - A u, computed on the fly at the 27 fine
// points of each coarse interior node (one kernel instead of two)
template <typename T>
__global__ void k_resid_restrict(const T* __restrict__ u, const T* __restrict__ f, T* __restrict__ fc, Dims df, Dims dc,
                                 T inv_h2)
{
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = 1 + blockIdx.z;
    if (I >= dc.nx || J >= dc.ny) return;
    const int Pf = df.nx * df.ny;
    const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * K;
    const int cols[3] = {(i0 == 0) ? df.nx - 1 : i0 - 1, i0, i0 + 1};
    const int rows[3] = {(j0 == 0) ? df.ny - 1 : j0 - 1, j0, j0 + 1};
    const T w[3] = {(T)0.25, (T)0.5, (T)0.25};
    T acc = (T)0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int k = k0 - 1 + a;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int j = rows[b];
            const int jp = (j + 1 == df.ny) ? 0 : j + 1, jm = (j == 0) ? df.ny - 1 : j - 1;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int i = cols[c];
                const int ip = (i + 1 == df.nx) ? 0 : i + 1, im = (i == 0) ? df.nx - 1 : i - 1;
                const int m = k * Pf + j * df.nx + i;
                const T sum = u[m - i + ip] + u[m - i + im] + u[k * Pf + jp * df.nx + i] + u[k * Pf + jm * df.nx + i] +
                              u[m + Pf] + u[m - Pf];
                acc += (w[a] * w[b] * w[c]) * (f[m] - ((T)6 * u[m] - sum) * inv_h2);
            }
        }
    }
    fc[K * dc.nx * dc.ny + J * dc.nx + I] = acc;
}

// trilinear interpolation of the coarse correction, added on the fine interior
template <typename T>
__global__ void k_prolong(T* __restrict__ uf, const T* __restrict__ uc, Dims df, Dims dc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = 1 + blockIdx.z;
    if (i >= df.nx || j >= df.ny) return;
    const int I0 = i >> 1, I1 = (i & 1) ? ((I0 + 1 == dc.nx) ? 0 : I0 + 1) : I0;
    const int J0 = j >> 1, J1 = (j & 1) ? ((J0 + 1 == dc.ny) ? 0 : J0 + 1) : J0;
    const int K0 = k >> 1, K1 = (k & 1) ? K0 + 1 : K0;
    const int Pc = dc.nx * dc.ny;
    const T* a0 = uc + K0 * Pc;
    const T* a1 = uc + K1 * Pc;
    // a coincident axis repeats its node, so the 1/8 weights give 1/2 or 1 per axis
    const T v = (T)0.125 * (a0[J0 * dc.nx + I0] + a0[J0 * dc.nx + I1] + a0[J1 * dc.nx + I0] + a0[J1 * dc.nx + I1] +
                            a1[J0 * dc.nx + I0] + a1[J0 * dc.nx + I1] + a1[J1 * dc.nx + I0] + a1[J1 * dc.nx + I1]);
    uf[k * df.nx * df.ny + j * df.nx + i] += v;
}

// coarsest level: red-black sweeps inside one block
template <typename T>
__global__ void k_coarse(T* __restrict__ u, const T* __restrict__ f, Dims d, T h2, int sweeps)
{
    const int half = d.nx / 2;
    const int total = half * d.ny * (d.nz - 1);
    const size_t P = (size_t)d.nx * d.ny;
    for (int s = 0; s < sweeps; ++s)
        for (int color = 0; color < 2; ++color) {
            for (int t = threadIdx.x; t < total; t += blockDim.x) {
                const int i2 = t % half;
                const int j = (t / half) % d.ny;
                const int k = 1 + t / (half * d.ny);
                const int i = 2 * i2 + ((j + k + color) & 1);
                const size_t n = nid(d, i, j, k);
                const int ip = (i + 1 == d.nx) ? 0 : i + 1, im = (i == 0) ? d.nx - 1 : i - 1;
                const int jp = (j + 1 == d.ny) ? 0 : j + 1, jm = (j == 0) ? d.ny - 1 : j - 1;
                const size_t row = n - i;
                const T sum = u[row + ip] + u[row + im] + u[nid(d, i, jp, k)] + u[nid(d, i, jm, k)] + u[n + P] +
                              u[n - P];
                u[n] = (sum + h2 * f[n]) * (T)(1.0 / 6.0);
            }
            __syncthreads();
        }
}

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double part[32];
    const int t = tid_flat(), nt = blockDim.x * blockDim.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = t & 31, w = t >> 5;
    if (lane == 0) part[w] = v;
    __syncthreads();
    v = (t < (nt + 31) / 32) ? part[t] : 0.0;
    if (w == 0)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// phi_out = phi + e on the interior (e may be null), r = f - A phi_out in FP64,
// stored as T; ||r||^2 accumulated into *norm2.  Thread (i, j) of interior
// plane k = 1 + blockIdx.z.
template <typename T>
__global__ void k_resid64(const double* __restrict__ phi, const T* __restrict__ e, const double* __restrict__ f,
                          double* __restrict__ phi_out, T* __restrict__ r, double* norm2, Dims d, double inv_h2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    double acc = 0.0;
    if (i < d.nx && j < d.ny) {
        const int P = d.nx * d.ny;
        const int ip = (i + 1 == d.nx) ? 0 : i + 1, im = (i == 0) ? d.nx - 1 : i - 1;
        const int jp = (j + 1 == d.ny) ? -j * d.nx : d.nx, jm = (j == 0) ? (d.ny - 1) * d.nx : -d.nx;
        // planes 1 + blockIdx.z, 1 + blockIdx.z + gridDim.z, ... (few blocks: few norm atomics)
        for (int k = 1 + blockIdx.z; k < d.nz; k += gridDim.z) {
            const int n = k * P + j * d.nx + i;
            const int row = n - i;
            const int nb[6] = {row + ip, row + im, n + jp, n + jm, n + P, n - P};
            double c = phi[n];
            double s = 0.0;
            if (e) {
                c += (double)e[n];
#pragma unroll
                for (int q = 0; q < 6; ++q) s += phi[nb[q]] + (double)e[nb[q]];
            } else {
#pragma unroll
                for (int q = 0; q < 6; ++q) s += phi[nb[q]];
            }
            if (phi_out) phi_out[n] = c;
            const double res = f[n] - (6.0 * c - s) * inv_h2;
            r[n] = (T)res;
            acc += res * res;
        }
    }
    acc = block_sum(acc);
    if (tid_flat() == 0) atomicAdd(norm2, acc);
}

// copy the electrode planes from phi to phi_out (the fused update writes only
// the interior)
__global__ void k_copy_planes(const double* __restrict__ phi, double* __restrict__ phi_out, Dims d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= d.nx || j >= d.ny) return;
    const int P = d.nx * d.ny;
    const int n = (blockIdx.z ? d.nz : 0) * P + j * d.nx + i;
    phi_out[n] = phi[n];
}

// f = rho_q * scale on every node; electrode values on both phi buffers;
// ||b||^2 with the electrode terms of the nodes next to the planes.  When
// vb_last (the lower electrode value of the previous solve) is given, the
// warm start moves by the change of the electrode ramp, (vb - vb_last)(1 - z/Lz),
// which the 7-point operator maps to zero: the starting residual then holds
// only the change of rho.
__global__ void k_rhs(const unsigned long long* __restrict__ rq, double scale, double* __restrict__ f,
                      double* __restrict__ phi, double* __restrict__ phi_alt, double vb, double vt, Dims d,
                      double inv_h2, double* norm2, const double* vb_last)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const double shift = vb_last ? vb - *vb_last : 0.0;
    double acc = 0.0;
    if (i < d.nx && j < d.ny)
        for (int k = blockIdx.z; k <= d.nz; k += gridDim.z) {
            const int n = (k * d.ny + j) * d.nx + i;
            const double fv = (double)(long long)rq[n] * scale;
            f[n] = fv;
            if (k == 0) { phi[n] = vb; phi_alt[n] = vb; }
            else if (k == d.nz) { phi[n] = vt; phi_alt[n] = vt; }
            else {
                if (shift != 0.0) phi[n] += shift * (1.0 - (double)k / (double)d.nz);
                double b = fv;
                if (k == 1) b += vb * inv_h2;
                if (k == d.nz - 1) b += vt * inv_h2;
                acc += b * b;
            }
        }
    acc = block_sum(acc);
    if (tid_flat() == 0) atomicAdd(norm2, acc);
}

__global__ void k_store(double* dst, double v) { *dst = v; }

// phi += e on the interior nodes
template <typename T>
__global__ void k_add(double* __restrict__ phi, const T* __restrict__ e, Dims d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= d.nx || j >= d.ny) return;
    const int n = ((1 + blockIdx.z) * d.ny + j) * d.nx + i;
    phi[n] += (double)e[n];
}

// electrode values at t = step * dt from the device step counter
__device__ __forceinline__ double bottom_potential(const SolveParams& sp, uint32_t step)
{
    const double t = (double)step * sp.dt;
    return sp.v_dc + sp.v_rf * sin((2.0 * kPI * sp.f_rf) * t + sp.phase);
}

// f = rho_q * scale; electrode values on phi; ||b||^2 added into norm[0];
// warm start moved by the change of the electrode ramp (as in k_rhs)
__global__ void k_rhs_dev(const unsigned long long* __restrict__ rq, double* __restrict__ f, double* __restrict__ phi,
                          Dims d, SolveParams sp, const uint32_t* step, double* norm2, const double* vb_last)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const double vb = bottom_potential(sp, *step), vt = sp.v_top;
    const double shift = vb - *vb_last;
    double acc = 0.0;
    if (i < d.nx && j < d.ny)
        for (int k = blockIdx.z; k <= d.nz; k += gridDim.z) {
            const int n = (k * d.ny + j) * d.nx + i;
            const double fv = (double)(long long)rq[n] * sp.scale;
            f[n] = fv;
            if (k == 0) phi[n] = vb;
            else if (k == d.nz) phi[n] = vt;
            else {
                if (shift != 0.0) phi[n] += shift * (1.0 - (double)k / (double)d.nz);
                double b = fv;
                if (k == 1) b += vb * sp.inv_h2;
                if (k == d.nz - 1) b += vt * sp.inv_h2;
                acc += b * b;
            }
        }
    acc = block_sum(acc);
    if (tid_flat() == 0) atomicAdd(norm2, acc);
}

// loop control of the graph solve: after each residual, decide whether to run
// another refinement iteration; record iterations, residual and non-convergence
__global__ void k_conv(double* norm, unsigned int* iters, double* res_out, int* flag, unsigned long long* total,
                       double tol2, int max_iters, int first, cudaGraphConditionalHandle h, double* vb_last,
                       SolveParams sp, const uint32_t* step)
{
    if (first) *vb_last = bottom_potential(sp, *step);
    const double b2 = norm[0], r2 = norm[1];
    const double target2 = tol2 * (b2 > 0.0 ? b2 : 1.0);
    unsigned int it = first ? 0u : *iters + 1u;
    *iters = it;
    if (!first) *total += 1ull;
    const bool ok = r2 <= target2;
    const bool finite = isfinite(r2);
    const bool more = !ok && finite && (int)it < max_iters;
    *res_out = b2 > 0.0 ? sqrt(r2 / b2) : sqrt(r2);
    if (!more && !ok) atomicCAS(flag, 0, finite ? (int)PIC_ENOTCONV : (int)PIC_ENONFINITE);
    norm[1] = 0.0;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// ---- the small levels of a V-cycle in one block --------------------------
constexpr int kTailMax = 8;

template <typename T>
struct TailLevels {
    int n;                        // levels in the tail (the last one is the coarsest)
    int nx[kTailMax], ny[kTailMax], nz[kTailMax];
    double h[kTailMax];
    T* u[kTailMax];
    T* f[kTailMax];
    T* r[kTailMax];
    const T* ainv;                // dense inverse of the coarsest level, or null
    int sweeps;                   // coarsest-level sweeps when there is no inverse
};

template <typename T>
__device__ void tail_rbgs(T* u, const T* f, Dims d, T h2, int color, bool zero)
{
    const int half = d.nx / 2;
    const int total = half * d.ny * (d.nz - 1);
    const int P = d.nx * d.ny;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int i2 = t % half;
        const int j = (t / half) % d.ny;
        const int k = 1 + t / (half * d.ny);
        const int i = 2 * i2 + ((j + k + color) & 1);
        const int n = (k * d.ny + j) * d.nx + i;
        if (zero) {
            u[n] = (h2 * f[n]) * (T)(1.0 / 6.0);
            continue;
        }
        const int ip = (i + 1 == d.nx) ? 0 : i + 1, im = (i == 0) ? d.nx - 1 : i - 1;
        const int jp = (j + 1 == d.ny) ? 0 : j + 1, jm = (j == 0) ? d.ny - 1 : j - 1;
        const int row = n - i;
        const T s = u[row + ip] + u[row + im] + u[(k * d.ny + jp) * d.nx + i] + u[(k * d.ny + jm) * d.nx + i] +
                    u[n + P] + u[n - P];
        u[n] = (s + h2 * f[n]) * (T)(1.0 / 6.0);
    }
    __syncthreads();
}

template <typename T>
__device__ void tail_resid(const T* u, const T* f, T* r, Dims d, T inv_h2)
{
    const int P = d.nx * d.ny;
    const int N = P * (d.nz + 1);
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const int k = n / P;
        if (k == 0 || k == d.nz) { r[n] = (T)0; continue; }
        const int i = n % d.nx, j = (n / d.nx) % d.ny;
        const int ip = (i + 1 == d.nx) ? 0 : i + 1, im = (i == 0) ? d.nx - 1 : i - 1;
        const int jp = (j + 1 == d.ny) ? 0 : j + 1, jm = (j == 0) ? d.ny - 1 : j - 1;
        const int row = n - i;
        const T s = u[row + ip] + u[row + im] + u[(k * d.ny + jp) * d.nx + i] + u[(k * d.ny + jm) * d.nx + i] +
                    u[n + P] + u[n - P];
        r[n] = f[n] - ((T)6 * u[n] - s) * inv_h2;
    }
    __syncthreads();
}

template <typename T>
__device__ void tail_restrict(const T* rf, T* fc, Dims df, Dims dc)
{
    const int P = dc.nx * dc.ny;
    const int N = P * (dc.nz + 1);
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const int K = n / P;
        if (K == 0 || K == dc.nz) { fc[n] = (T)0; continue; }
        const int I = n % dc.nx, J = (n / dc.nx) % dc.ny;
        T acc = (T)0;
        for (int dk = -1; dk <= 1; ++dk) {
            const T wk = dk == 0 ? (T)0.5 : (T)0.25;
            for (int dj = -1; dj <= 1; ++dj) {
                const T wj = dj == 0 ? (T)0.5 : (T)0.25;
                const int j = (2 * J + dj + df.ny) % df.ny;
                for (int di = -1; di <= 1; ++di) {
                    const T wi = di == 0 ? (T)0.5 : (T)0.25;
                    const int i = (2 * I + di + df.nx) % df.nx;
                    acc += (wk * wj * wi) * rf[((2 * K + dk) * df.ny + j) * df.nx + i];
                }
            }
        }
        fc[n] = acc;
    }
    __syncthreads();
}

// restriction of the residual f - A u computed on the fly at the 27 fine points
template <typename T>
__device__ void tail_resid_restrict(const T* u, const T* f, T* fc, Dims df, Dims dc, T inv_h2)
{
    const int P = dc.nx * dc.ny;
    const int N = P * (dc.nz - 1);
    const int Pf = df.nx * df.ny;
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        const int n = P + t;
        const int K = n / P;
        const int I = n % dc.nx, J = (n / dc.nx) % dc.ny;
        T acc = (T)0;
        for (int dk = -1; dk <= 1; ++dk) {
            const T wk = dk == 0 ? (T)0.5 : (T)0.25;
            const int k = 2 * K + dk;
            for (int dj = -1; dj <= 1; ++dj) {
                const T wj = dj == 0 ? (T)0.5 : (T)0.25;
                const int j = (2 * J + dj + df.ny) % df.ny;
                const int jp = (j + 1 == df.ny) ? 0 : j + 1, jm = (j == 0) ? df.ny - 1 : j - 1;
                for (int di = -1; di <= 1; ++di) {
                    const T wi = di == 0 ? (T)0.5 : (T)0.25;
                    const int i = (2 * I + di + df.nx) % df.nx;
                    const int ip = (i + 1 == df.nx) ? 0 : i + 1, im = (i == 0) ? df.nx - 1 : i - 1;
                    const int m = k * Pf + j * df.nx + i;
                    const T sum = u[m - i + ip] + u[m - i + im] + u[k * Pf + jp * df.nx + i] +
                                  u[k * Pf + jm * df.nx + i] + u[m + Pf] + u[m - Pf];
                    acc += (wk * wj * wi) * (f[m] - ((T)6 * u[m] - sum) * inv_h2);
                }
            }
        }
        fc[n] = acc;
    }
    __syncthreads();
}

template <typename T>
__device__ void tail_prolong(T* uf, const T* uc, Dims df, Dims dc)
{
    const int P = df.nx * df.ny;
    const int N = P * (df.nz + 1);
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const int k = n / P;
        if (k == 0 || k == df.nz) continue;
        const int i = n % df.nx, j = (n / df.nx) % df.ny;
        const int I0 = i / 2, I1 = (i & 1) ? (i / 2 + 1) % dc.nx : I0;
        const int J0 = j / 2, J1 = (j & 1) ? (j / 2 + 1) % dc.ny : J0;
        const int K0 = k / 2, K1 = (k & 1) ? k / 2 + 1 : K0;
        const int Pc = dc.nx * dc.ny;
        // each axis: weights (1/2, 1/2) between two coarse nodes, or (1) on a coincident one
        const T v = (T)0.125 * (uc[K0 * Pc + J0 * dc.nx + I0] + uc[K0 * Pc + J0 * dc.nx + I1] +
                                uc[K0 * Pc + J1 * dc.nx + I0] + uc[K0 * Pc + J1 * dc.nx + I1] +
                                uc[K1 * Pc + J0 * dc.nx + I0] + uc[K1 * Pc + J0 * dc.nx + I1] +
                                uc[K1 * Pc + J1 * dc.nx + I0] + uc[K1 * Pc + J1 * dc.nx + I1]);
        uf[n] += v;
    }
    __syncthreads();
}

// The lower part of a V(2,2) cycle in one block with every tail level held in
// shared memory: pre-smoothing from a zero guess, residual restricted to the
// next level, the coarsest solve, prolongation and post-smoothing.  Global
// memory is touched only to read the first tail level's right-hand side and
// write back its correction.
template <typename T>
__global__ void __launch_bounds__(1024) k_vcycle_tail(const TailLevels<T> L)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T* su[kTailMax];
    T* sf[kTailMax];
    {
        T* p = reinterpret_cast<T*>(smem);
        for (int l = 0; l < L.n; ++l) {
            const int nodes = L.nx[l] * L.ny[l] * (L.nz[l] + 1);
            su[l] = p; p += nodes;
            sf[l] = p; p += nodes;
        }
        // corrections start at zero (electrode planes stay zero); first rhs from global
        for (int l = 0; l < L.n; ++l) {
            const int nodes = L.nx[l] * L.ny[l] * (L.nz[l] + 1);
            for (int t = threadIdx.x; t < nodes; t += blockDim.x) {
                su[l][t] = (T)0;
                sf[l][t] = l == 0 ? L.f[0][t] : (T)0;
            }
        }
        __syncthreads();
    }
    for (int l = 0; l + 1 < L.n; ++l) {
        const Dims d{L.nx[l], L.ny[l], L.nz[l]};
        const T h2 = (T)(L.h[l] * L.h[l]);
        tail_rbgs<T>(su[l], sf[l], d, h2, 0, true);
        tail_rbgs<T>(su[l], sf[l], d, h2, 1, false);
        tail_rbgs<T>(su[l], sf[l], d, h2, 0, false);
        tail_rbgs<T>(su[l], sf[l], d, h2, 1, false);
        tail_resid_restrict<T>(su[l], sf[l], sf[l + 1], d, Dims{L.nx[l + 1], L.ny[l + 1], L.nz[l + 1]},
                               (T)(1.0 / (L.h[l] * L.h[l])));
    }
    {
        const int c = L.n - 1;
        const Dims d{L.nx[c], L.ny[c], L.nz[c]};
        const int P = d.nx * d.ny, n = P * (d.nz - 1);
        if (L.ainv) {
            for (int m = threadIdx.x; m < n; m += blockDim.x) {
                const T* row = L.ainv + (size_t)m * n;
                T acc = (T)0;
                for (int q = 0; q < n; ++q) acc += row[q] * sf[c][P + q];
                su[c][P + m] = acc;
            }
            __syncthreads();
        } else {
            const T h2 = (T)(L.h[c] * L.h[c]);
            for (int s = 0; s < L.sweeps; ++s) {
                tail_rbgs<T>(su[c], sf[c], d, h2, 0, s == 0);
                tail_rbgs<T>(su[c], sf[c], d, h2, 1, false);
            }
        }
    }
    for (int l = L.n - 2; l >= 0; --l) {
        const Dims d{L.nx[l], L.ny[l], L.nz[l]};
        const T h2 = (T)(L.h[l] * L.h[l]);
        tail_prolong<T>(su[l], su[l + 1], d, Dims{L.nx[l + 1], L.ny[l + 1], L.nz[l + 1]});
        tail_rbgs<T>(su[l], sf[l], d, h2, 0, false);
        tail_rbgs<T>(su[l], sf[l], d, h2, 1, false);
        tail_rbgs<T>(su[l], sf[l], d, h2, 0, false);
        tail_rbgs<T>(su[l], sf[l], d, h2, 1, false);
    }
    const int nodes0 = L.nx[0] * L.ny[0] * (L.nz[0] + 1);
    for (int t = threadIdx.x; t < nodes0; t += blockDim.x) L.u[0][t] = su[0][t];
}

template <typename T>
size_t tail_smem(const pic_ctx* c, int l0)
{
    size_t b = 0;
    for (size_t l = (size_t)l0; l < c->mg.size(); ++l) b += 2 * sizeof(T) * c->mg[l].nodes;
    return b;
}

int blocks(size_t n) { return grid_for((int64_t)n, 256, 152 * 8); }

// grid for kernels that reduce a norm: (x, y) blocks of a plane and just enough
// z blocks (each looping over planes) to fill the GPU a few times
inline Grid3 grid_norm(int nx, int ny, int planes)
{
    Grid3 g = grid3(nx, ny, 1);
    const int per_plane = (int)(g.grid.x * g.grid.y);
    const int zb = std::max(1, std::min(planes, (152 * 4 + per_plane - 1) / per_plane));
    g.grid.z = (unsigned)zb;
    return g;
}

template <typename T>
void run_rbgs(cudaStream_t s, T* u, const T* f, Dims d, T h2, int color, int zero)
{
    const Grid3 g = grid3(d.nx / 2, d.ny, d.nz - 1);
    k_rbgs<T><<<g.grid, g.block, 0, s>>>(u, f, d, h2, color, zero);
}
template <typename T>
void run_resid(cudaStream_t s, const T* u, const T* f, T* r, Dims d, T inv_h2)
{
    const Grid3 g = grid3(d.nx, d.ny, d.nz - 1);
    k_resid<T><<<g.grid, g.block, 0, s>>>(u, f, r, d, inv_h2);
}
template <typename T>
void run_restrict(cudaStream_t s, const T* rf, T* fc, Dims df, Dims dc)
{
    const Grid3 g = grid3(dc.nx, dc.ny, dc.nz - 1);
    k_restrict<T><<<g.grid, g.block, 0, s>>>(rf, fc, df, dc);
}
template <typename T>
void run_resid_restrict(cudaStream_t s, const T* u, const T* f, T* fc, Dims df, Dims dc, T inv_h2)
{
    const Grid3 g = grid3(dc.nx, dc.ny, dc.nz - 1);
    k_resid_restrict<T><<<g.grid, g.block, 0, s>>>(u, f, fc, df, dc, inv_h2);
}
template <typename T>
void run_prolong(cudaStream_t s, T* uf, const T* uc, Dims df, Dims dc)
{
    const Grid3 g = grid3(df.nx, df.ny, df.nz - 1);
    k_prolong<T><<<g.grid, g.block, 0, s>>>(uf, uc, df, dc);
}
template <typename T>
void run_resid64(cudaStream_t s, const double* phi, const T* e, const double* f, double* phi_out, T* r, double* norm2,
                 Dims d, double inv_h2)
{
    const Grid3 g = grid_norm(d.nx, d.ny, d.nz - 1);
    k_resid64<T><<<g.grid, g.block, 0, s>>>(phi, e, f, phi_out, r, norm2, d, inv_h2);
    if (phi_out) {
        const Grid3 g2 = grid3(d.nx, d.ny, 2);
        k_copy_planes<<<g2.grid, g2.block, 0, s>>>(phi, phi_out, d);
    }
}

template <typename T>
void vcycle(pic_ctx* c, int l)
{
    const int nl = (int)c->mg.size();
    if (l >= c->mg_tail) {
        // every level from here down runs in one block
        TailLevels<T> t{};
        t.n = nl - l;
        for (int q = 0; q < t.n; ++q) {
            const MGLevel& L = c->mg[l + q];
            t.nx[q] = L.nx; t.ny[q] = L.ny; t.nz[q] = L.nz; t.h[q] = L.h;
            t.u[q] = (T*)L.u; t.f[q] = (T*)L.f; t.r[q] = (T*)L.r;
        }
        const MGLevel& C = c->mg.back();
        const int n = C.nx * C.ny * (C.nz - 1);
        t.ainv = (const T*)c->coarse_inv;
        const int m = std::max(std::max(C.nx, C.ny), C.nz);
        t.sweeps = std::min(4 * m * m + 16, 2000);
        (void)n;
        k_vcycle_tail<T><<<1, 1024, tail_smem<T>(c, l), c->stream>>>(t);
        c->launches += 1;
        return;
    }
    MGLevel& L = c->mg[l];
    const Dims d{L.nx, L.ny, L.nz};
    const T h2 = (T)(L.h * L.h);
    T* u = (T*)L.u;
    T* f = (T*)L.f;
    // pre-smoothing from a zero guess: the first colour-0 pass needs no neighbours
    for (int s = 0; s < kPre; ++s)
        for (int color = 0; color < 2; ++color) run_rbgs<T>(c->stream, u, f, d, h2, color, s == 0 && color == 0);
    MGLevel& C = c->mg[l + 1];
    const Dims dc{C.nx, C.ny, C.nz};
    run_resid_restrict<T>(c->stream, u, f, (T*)C.f, d, dc, (T)(1.0 / (L.h * L.h)));
    c->launches += 2 * kPre + 1;
    vcycle<T>(c, l + 1);
    run_prolong<T>(c->stream, u, (const T*)C.u, d, dc);
    c->launches += 1 + 2 * kPost;
    for (int s = 0; s < kPost; ++s)
        for (int color = 0; color < 2; ++color) run_rbgs<T>(c->stream, u, f, d, h2, color, 0);
}

template <typename T>
pic_status solve_t(pic_ctx* c, double tol, int max_iters, int* iters, double* res)
{
    const Dims d{c->nx, c->ny, c->nz};
    const double inv_h2 = 1.0 / (c->dx * c->dx);
    MGLevel& L0 = c->mg[0];
    double h_norm[2];
    // initial residual (phi unchanged)
    cudaMemsetAsync(c->d_norm + 1, 0, sizeof(double), c->stream);
    run_resid64<T>(c->stream, c->phi, (const T*)nullptr, c->f64, nullptr, (T*)L0.f, c->d_norm + 1, d, inv_h2);
    c->launches += 1;
    if (!PIC_CUDA_OK(cudaMemcpyAsync(h_norm, c->d_norm, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream)) ||
        !PIC_CUDA_OK(cudaStreamSynchronize(c->stream)))
        return PIC_ECUDA;
    const double bn = std::sqrt(h_norm[0]);
    double rn = std::sqrt(h_norm[1]);
    const double target = tol * (bn > 0.0 ? bn : 1.0);
    int it = 0;
    while (!(rn <= target) && it < max_iters) {
        if (!std::isfinite(rn)) break;
        vcycle<T>(c, 0);
        cudaMemsetAsync(c->d_norm + 1, 0, sizeof(double), c->stream);
        run_resid64<T>(c->stream, c->phi, (const T*)L0.u, c->f64, c->phi_alt, (T*)L0.f, c->d_norm + 1, d, inv_h2);
        c->launches += 2;
        std::swap(c->phi, c->phi_alt);
        if (!PIC_CUDA_OK(cudaMemcpyAsync(h_norm + 1, c->d_norm + 1, sizeof(double), cudaMemcpyDeviceToHost,
                                         c->stream)) ||
            !PIC_CUDA_OK(cudaStreamSynchronize(c->stream)))
            return PIC_ECUDA;
        rn = std::sqrt(h_norm[1]);
        ++it;
    }
    if (iters) *iters = it;
    const double rel = bn > 0.0 ? rn / bn : rn;
    if (res) *res = rel;
    c->last_iters = it;
    c->last_res = rel;
    if (!std::isfinite(rn)) return PIC_ENONFINITE;
    return rn <= target ? PIC_OK : PIC_ENOTCONV;
}

// One refinement iteration (the body of the graph's while loop):
// V-cycle on A e = r, phi += e, r = f - A phi, loop decision.
template <typename T>
void enqueue_iteration(pic_ctx* c, double tol, int max_iters, cudaGraphConditionalHandle h)
{
    const Dims d{c->nx, c->ny, c->nz};
    vcycle<T>(c, 0);
    const Grid3 g = grid3(d.nx, d.ny, d.nz - 1);
    k_add<T><<<g.grid, g.block, 0, c->stream>>>(c->phi, (const T*)c->mg[0].u, d);
    run_resid64<T>(c->stream, c->phi, (const T*)nullptr, c->f64, nullptr, (T*)c->mg[0].f, c->d_norm + 1, d,
                   1.0 / (c->dx * c->dx));
    k_conv<<<1, 1, 0, c->stream>>>(c->d_norm, c->d_iters, c->d_res, c->d_solve_flag, c->d_iter_total, tol * tol,
                                   max_iters, 0, h, c->d_vb_last, c->sp, c->d_step);
    c->launches += 3;
}

// Head of the graph solve: rhs from rho with the electrode values of the
// device step, the starting residual, and the first loop decision.
template <typename T>
void enqueue_head(pic_ctx* c, double tol, int max_iters, cudaGraphConditionalHandle h)
{
    const Dims d{c->nx, c->ny, c->nz};
    cudaMemsetAsync(c->d_norm, 0, 2 * sizeof(double), c->stream);
    const Grid3 g = grid_norm(d.nx, d.ny, d.nz + 1);
    k_rhs_dev<<<g.grid, g.block, 0, c->stream>>>(c->rq, c->f64, c->phi, d, c->sp, c->d_step, c->d_norm,
                                                c->d_vb_last);
    run_resid64<T>(c->stream, c->phi, (const T*)nullptr, c->f64, nullptr, (T*)c->mg[0].f, c->d_norm + 1, d,
                   1.0 / (c->dx * c->dx));
    k_conv<<<1, 1, 0, c->stream>>>(c->d_norm, c->d_iters, c->d_res, c->d_solve_flag, c->d_iter_total, tol * tol,
                                   max_iters, 1, h, c->d_vb_last, c->sp, c->d_step);
    c->launches += 3;
}

}  // namespace

void enqueue_solve_head(pic_ctx* c, double tol, int max_iters, cudaGraphConditionalHandle h)
{
    if (c->prec == PIC_MIXED) enqueue_head<float>(c, tol, max_iters, h);
    else enqueue_head<double>(c, tol, max_iters, h);
}

void enqueue_solve_iteration(pic_ctx* c, double tol, int max_iters, cudaGraphConditionalHandle h)
{
    if (c->prec == PIC_MIXED) enqueue_iteration<float>(c, tol, max_iters, h);
    else enqueue_iteration<double>(c, tol, max_iters, h);
}

pic_status mg_setup(pic_ctx* c)
{
    const size_t tsz = c->prec == PIC_MIXED ? sizeof(float) : sizeof(double);
    int nx = c->nx, ny = c->ny, nz = c->nz;
    double h = c->dx;
    c->mg.clear();
    while (true) {
        MGLevel L;
        L.nx = nx; L.ny = ny; L.nz = nz; L.h = h;
        L.nodes = (size_t)nx * ny * (nz + 1);
        L.u = dev_alloc(c, tsz * L.nodes);
        L.f = dev_alloc(c, tsz * L.nodes);
        L.r = dev_alloc(c, tsz * L.nodes);
        if (!L.u || !L.f || !L.r) return PIC_ENOMEM;
        // electrode planes of the corrections stay zero: they are never written
        if (cudaMemset(L.u, 0, tsz * L.nodes) != cudaSuccess || cudaMemset(L.f, 0, tsz * L.nodes) != cudaSuccess ||
            cudaMemset(L.r, 0, tsz * L.nodes) != cudaSuccess)
            return PIC_ECUDA;
        c->mg.push_back(L);
        const bool can = nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0 && nx >= 4 && ny >= 4 && nz >= 4 &&
                         (nx / 2) % 2 == 0 && (ny / 2) % 2 == 0;
        if (!can) break;
        nx /= 2; ny /= 2; nz /= 2; h *= 2.0;
    }
    // the smallest levels (each at most kTailNodes nodes, at most kTailMax of them,
    // together at most kTailSmem bytes of u and f) run in one block from shared
    // memory; larger levels are faster as grid-wide launches
    c->mg_tail = (int)c->mg.size() - 1;
    auto smem_from = [&](int l0) {
        size_t b = 0;
        for (size_t l = (size_t)l0; l < c->mg.size(); ++l) b += 2 * tsz * c->mg[l].nodes;
        return b;
    };
    while (c->mg_tail > 0 && smem_from(c->mg_tail - 1) <= kTailSmem && c->mg[c->mg_tail - 1].nodes <= kTailNodes &&
           (int)c->mg.size() - (c->mg_tail - 1) <= kTailMax)
        --c->mg_tail;
    {
        const cudaError_t e = c->prec == PIC_MIXED
            ? cudaFuncSetAttribute(k_vcycle_tail<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmem)
            : cudaFuncSetAttribute(k_vcycle_tail<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmem);
        if (e != cudaSuccess) return PIC_ECUDA;
    }
    // exact inverse of the coarsest operator (6 u - neighbour sum) / h^2 with
    // zero values on the electrode planes, by Gauss-Jordan elimination
    const MGLevel& L = c->mg.back();
    const int P = L.nx * L.ny, n = P * (L.nz - 1);
    c->coarse_inv = nullptr;
    if (n <= kMaxDense && n > 0) {
        std::vector<double> a((size_t)n * n, 0.0), inv((size_t)n * n, 0.0);
        const double ih2 = 1.0 / (L.h * L.h);
        for (int k = 1; k < L.nz; ++k)
            for (int j = 0; j < L.ny; ++j)
                for (int i = 0; i < L.nx; ++i) {
                    const int m = (k - 1) * P + j * L.nx + i;
                    a[(size_t)m * n + m] += 6.0 * ih2;
                    const int nb[6][3] = {{(i + 1) % L.nx, j, k}, {(i + L.nx - 1) % L.nx, j, k},
                                          {i, (j + 1) % L.ny, k}, {i, (j + L.ny - 1) % L.ny, k},
                                          {i, j, k + 1}, {i, j, k - 1}};
                    for (auto& q : nb) {
                        if (q[2] == 0 || q[2] == L.nz) continue;
                        a[(size_t)m * n + (q[2] - 1) * P + q[1] * L.nx + q[0]] -= ih2;
                    }
                }
        for (int m = 0; m < n; ++m) inv[(size_t)m * n + m] = 1.0;
        for (int col = 0; col < n; ++col) {
            int piv = col;
            for (int r = col + 1; r < n; ++r)
                if (std::fabs(a[(size_t)r * n + col]) > std::fabs(a[(size_t)piv * n + col])) piv = r;
            if (piv != col)
                for (int q = 0; q < n; ++q) {
                    std::swap(a[(size_t)piv * n + q], a[(size_t)col * n + q]);
                    std::swap(inv[(size_t)piv * n + q], inv[(size_t)col * n + q]);
                }
            const double dg = a[(size_t)col * n + col];
            for (int q = 0; q < n; ++q) { a[(size_t)col * n + q] /= dg; inv[(size_t)col * n + q] /= dg; }
            for (int r = 0; r < n; ++r) {
                if (r == col) continue;
                const double fct = a[(size_t)r * n + col];
                if (fct == 0.0) continue;
                for (int q = 0; q < n; ++q) {
                    a[(size_t)r * n + q] -= fct * a[(size_t)col * n + q];
                    inv[(size_t)r * n + q] -= fct * inv[(size_t)col * n + q];
                }
            }
        }
        void* d = dev_alloc(c, tsz * (size_t)n * n);
        if (!d) return PIC_ENOMEM;
        cudaError_t e;
        if (c->prec == PIC_MIXED) {
            std::vector<float> f32(inv.begin(), inv.end());
            e = cudaMemcpy(d, f32.data(), sizeof(float) * f32.size(), cudaMemcpyHostToDevice);
        } else {
            e = cudaMemcpy(d, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return PIC_ECUDA;
        c->coarse_inv = d;
    }
    return PIC_OK;
}

void launch_rhs(pic_ctx* c, double scale, double v_bot, double v_top, bool)
{
    const Dims d{c->nx, c->ny, c->nz};
    cudaMemsetAsync(c->d_norm, 0, sizeof(double), c->stream);
    const Grid3 g = grid_norm(d.nx, d.ny, d.nz + 1);
    k_rhs<<<g.grid, g.block, 0, c->stream>>>(c->rq, scale, c->f64, c->phi, c->phi_alt, v_bot, v_top, d,
                                            1.0 / (c->dx * c->dx), c->d_norm, c->d_vb_last);
    k_store<<<1, 1, 0, c->stream>>>(c->d_vb_last, v_bot);
    c->launches += 2;
}

pic_status mg_solve(pic_ctx* c, double, double, double tol, int max_iters, int* iters, double* res)
{
    if (c->prec == PIC_MIXED) return solve_t<float>(c, tol, max_iters, iters, res);
    return solve_t<double>(c, tol, max_iters, iters, res);
}

}  // namespace pic

// ---------------------------------------------------------------------------
// pic_solve_noalloc: the same multigrid solve for callers that cannot allocate
// device memory.  Its whole working set (second potential buffer, right-hand
// side, norms and every level's u, f, r) lives in one file-scope device array
// of fixed size, which each GPU that loads the library holds until exit.
namespace pic {
namespace {

constexpr size_t kNaMaxNodes = 131072;       // largest fine mesh, in nodes
constexpr size_t kNaAlign = 256;
// phi_alt + f (16 B/node) + three level arrays summing to at most 4/3 of the
// fine nodes in doubles (32 B/node) + norms + per-array alignment padding
constexpr size_t kNaBytes = kNaMaxNodes * 48 + 64 * kNaAlign + 4096;
constexpr int kNaMaxDevices = 64;
constexpr int kNaMaxLevels = 24;

static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

std::mutex g_na_mu;
unsigned char* g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the array's name is only a host-side stand-in in host code).
pic_status na_scratch(unsigned char** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return PIC_ECUDA;
    if (dev < 0 || dev >= kNaMaxDevices) return PIC_EINVAL;
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return PIC_ECUDA;
        g_na_ptr[dev] = (unsigned char*)p;
    }
    *out = g_na_ptr[dev];
    return PIC_OK;
}

struct NaCtx {
    MGLevel lv[kNaMaxLevels];
    int nl;
    cudaStream_t s;
};

template <typename T>
void na_vcycle(NaCtx& c, int l)
{
    MGLevel& L = c.lv[l];
    const Dims d{L.nx, L.ny, L.nz};
    const T h2 = (T)(L.h * L.h);
    T* u = (T*)L.u;
    T* f = (T*)L.f;
    cudaMemsetAsync(u, 0, sizeof(T) * L.nodes, c.s);
    if (l + 1 == c.nl) {
        const int m = std::max(std::max(L.nx, L.ny), L.nz);
        k_coarse<T><<<1, 1024, 0, c.s>>>(u, f, d, h2, std::min(4 * m * m + 16, 2000));
        return;
    }
    const size_t half = (size_t)(L.nx / 2) * L.ny * (L.nz - 1);
    for (int s = 0; s < 2; ++s)
        for (int color = 0; color < 2; ++color) run_rbgs<T>(c.s, u, f, d, h2, color, 0);
    run_resid<T>(c.s, u, f, (T*)L.r, d, (T)(1.0 / (L.h * L.h)));
    MGLevel& C = c.lv[l + 1];
    const Dims dc{C.nx, C.ny, C.nz};
    run_restrict<T>(c.s, (const T*)L.r, (T*)C.f, d, dc);
    na_vcycle<T>(c, l + 1);
    run_prolong<T>(c.s, u, (const T*)C.u, d, dc);
    for (int s = 0; s < 2; ++s)
        for (int color = 0; color < 2; ++color) run_rbgs<T>(c.s, u, f, d, h2, color, 0);
}

template <typename T>
pic_status na_solve(NaCtx& c, double* phi_user, double* phi_alt, const double* f64, double* norm, Dims d,
                    double dx, double tol, int max_iters, int* iters, double* res)
{
    const double inv_h2 = 1.0 / (dx * dx);
    const size_t nodes = (size_t)d.nx * d.ny * (d.nz + 1);
    double h_norm[2];
    double* phi = phi_user;
    double* alt = phi_alt;
    cudaMemsetAsync(norm + 1, 0, sizeof(double), c.s);
    run_resid64<T>(c.s, phi, (const T*)nullptr, f64, nullptr, (T*)c.lv[0].f, norm + 1, d, inv_h2);
    if (cudaMemcpyAsync(h_norm, norm, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
        cudaStreamSynchronize(c.s) != cudaSuccess)
        return PIC_ECUDA;
    const double bn = std::sqrt(h_norm[0]);
    double rn = std::sqrt(h_norm[1]);
    const double target = tol * (bn > 0.0 ? bn : 1.0);
    int it = 0;
    while (!(rn <= target) && it < max_iters && std::isfinite(rn)) {
        na_vcycle<T>(c, 0);
        cudaMemsetAsync(norm + 1, 0, sizeof(double), c.s);
        run_resid64<T>(c.s, phi, (const T*)c.lv[0].u, f64, alt, (T*)c.lv[0].f, norm + 1, d, inv_h2);
        std::swap(phi, alt);
        if (cudaMemcpyAsync(h_norm + 1, norm + 1, sizeof(double), cudaMemcpyDeviceToHost, c.s) != cudaSuccess ||
            cudaStreamSynchronize(c.s) != cudaSuccess)
            return PIC_ECUDA;
        rn = std::sqrt(h_norm[1]);
        ++it;
    }
    // the last update may sit in the scratch buffer: return it in the caller's array
    if (phi != phi_user &&
        (cudaMemcpyAsync(phi_user, phi, sizeof(double) * nodes, cudaMemcpyDeviceToDevice, c.s) != cudaSuccess ||
         cudaStreamSynchronize(c.s) != cudaSuccess))
        return PIC_ECUDA;
    if (iters) *iters = it;
    if (res) *res = bn > 0.0 ? rn / bn : rn;
    if (!std::isfinite(rn)) return PIC_ENONFINITE;
    return rn <= target ? PIC_OK : PIC_ENOTCONV;
}

}  // namespace
}  // namespace pic

extern "C" pic_status pic_solve_noalloc(int32_t nx, int32_t ny, int32_t nz, double dx, const int64_t* rho_q_dev,
                                        double scale, double v_bot, double v_top, double* phi_dev, int32_t prec,
                                        double tol, int32_t max_iters, int32_t* iterations, double* rel_residual,
                                        void* cuda_stream)
{
    using namespace pic;
    if (nx < 4 || ny < 4 || nz < 2 || nx % 2 || ny % 2 || !(dx > 0.0) || !rho_q_dev || !phi_dev ||
        (prec != PIC_FP64 && prec != PIC_MIXED) || !(tol > 0.0) || max_iters < 1) {
        set_global_error("pic_solve_noalloc: invalid mesh, pointer, precision, tolerance or iteration limit");
        return PIC_EINVAL;
    }
    const size_t nodes = (size_t)nx * ny * (nz + 1);
    if (nodes > kNaMaxNodes) {
        set_global_error("pic_solve_noalloc: mesh has more than 131072 nodes (nx*ny*(nz+1)), the fixed scratch "
                         "limit; use pic_init/pic_solve for larger meshes");
        return PIC_EINVAL;
    }
    unsigned char* base = nullptr;
    pic_status st = na_scratch(&base);
    if (st != PIC_OK) {
        set_global_error("pic_solve_noalloc: could not look up the scratch array on the current device");
        return st;
    }
    // carve the scratch: phi_alt, f, norms, then the level arrays
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        void* p = base + off;
        off += (bytes + kNaAlign - 1) / kNaAlign * kNaAlign;
        return p;
    };
    double* phi_alt = (double*)take(sizeof(double) * nodes);
    double* f64 = (double*)take(sizeof(double) * nodes);
    double* norm = (double*)take(4 * sizeof(double));
    NaCtx c;
    c.s = (cudaStream_t)cuda_stream;
    c.nl = 0;
    const size_t tsz = prec == PIC_MIXED ? sizeof(float) : sizeof(double);
    int lx = nx, ly = ny, lz = nz;
    double h = dx;
    while (c.nl < kNaMaxLevels) {
        MGLevel& L = c.lv[c.nl++];
        L.nx = lx; L.ny = ly; L.nz = lz; L.h = h;
        L.nodes = (size_t)lx * ly * (lz + 1);
        L.u = take(tsz * L.nodes);
        L.f = take(tsz * L.nodes);
        L.r = take(tsz * L.nodes);
        const bool can = lx % 4 == 0 && ly % 4 == 0 && lz % 2 == 0 && lz >= 4;
        if (!can) break;
        lx /= 2; ly /= 2; lz /= 2; h *= 2.0;
    }
    if (off > kNaBytes) {
        set_global_error("pic_solve_noalloc: scratch layout exceeds the fixed array");
        return PIC_EINVAL;
    }
    // rhs from the fixed-point charge; electrode values on both potential buffers
    const Dims d{nx, ny, nz};
    cudaMemsetAsync(norm, 0, sizeof(double), c.s);
    const Grid3 g = grid_norm(nx, ny, nz + 1);
    k_rhs<<<g.grid, g.block, 0, c.s>>>((const unsigned long long*)rho_q_dev, scale, f64, phi_dev, phi_alt, v_bot,
                                      v_top, d, 1.0 / (dx * dx), norm, (const double*)nullptr);
    int it = 0;
    double res = 0.0;
    st = prec == PIC_MIXED ? na_solve<float>(c, phi_dev, phi_alt, f64, norm, d, dx, tol, max_iters, &it, &res)
                           : na_solve<double>(c, phi_dev, phi_alt, f64, norm, d, dx, tol, max_iters, &it, &res);
    if (iterations) *iterations = it;
    if (rel_residual) *rel_residual = res;
    if (st == PIC_ECUDA) set_global_error("pic_solve_noalloc: a CUDA call failed");
    else if (st == PIC_ENOTCONV) set_global_error("pic_solve_noalloc: tolerance not reached in max_iters");
    else if (st == PIC_ENONFINITE) set_global_error("pic_solve_noalloc: non-finite residual");
    return st;
}

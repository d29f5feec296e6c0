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
// doubling), the levels from a small one down in one thread-block cluster
// (an exact Fourier-Thomas solve of the first level that fits, or sweeps).
// The large grid-wide levels store u and f red-black split (lix), and their
// half-sweeps, red residuals and prolongation run as column kernels over node
// pairs, plane after plane; the mixed refinement keeps phi and f as two-float
// sums (double-float arithmetic).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include <cooperative_groups.h>

#include "pic_internal.cuh"

#ifndef PIC_MG_PRE
#define PIC_MG_PRE 2
#endif
#ifndef PIC_MG_POST
#define PIC_MG_POST 2
#endif
#ifndef PIC_MG_CLUSTER
#define PIC_MG_CLUSTER 16      // largest cluster (CTAs) for the small levels
#endif
#ifndef PIC_MG_CLUSTER_FROM
#define PIC_MG_CLUSTER_FROM 2  // first level that may run in the cluster
#endif
#ifndef PIC_PDL
#define PIC_PDL 1              // programmatic dependent launch between solver kernels
#endif
#ifndef PIC_MG_EXACT
#define PIC_MG_EXACT 1         // solve the first level that fits one cluster exactly
#endif
#ifndef PIC_MG_EXACT_MAXNODES
#define PIC_MG_EXACT_MAXNODES 32768  // largest level solved exactly (Fourier transforms cost grows as n^1.5)
#endif
#ifndef PIC_NORM_BLOCKS
#define PIC_NORM_BLOCKS 1216   // blocks of the plane-looping kernels that reduce a norm
#endif
#ifndef PIC_MG_CL_THREADS
#define PIC_MG_CL_THREADS 512  // threads per CTA of the cluster
#endif

namespace pic {
namespace {

namespace cg = cooperative_groups;

constexpr int kPre = PIC_MG_PRE;         // pre-smoothing sweeps of a V-cycle
constexpr int kPost = PIC_MG_POST;       // post-smoothing sweeps

struct Dims {
    int nx, ny, nz;
    int half = 0;   // > 0: the level's u and f are split by colour (red-black layout)
};

// Red-black layout of a level (nx even): the red nodes (i + j + k even) in
// the first half of the array, the black in the second, node n at n / 2 of
// its half (n and n + 1 of a row pair always differ in colour).  A half-sweep
// then reads one colour's half of u and f and the other colour's half of u,
// instead of every line of both.  half == 0: natural order.
__device__ __forceinline__ int lix(const Dims& d, int n, int colour)
{
    return d.half ? (colour ? d.half : 0) + (n >> 1) : n;
}

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

// Programmatic dependent launch: the solver's kernels are queued with the
// programmatic-serialization attribute, so the next kernel's blocks can be
// scheduled while this one drains.  Each kernel waits for its predecessor's
// completion (and memory) before touching anything, in every thread, so the
// ordering stays transitive; it then lets its own successor launch.
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch_pdl_smem(cudaStream_t s, dim3 grid, dim3 block, size_t smem, void (*kernel)(KArgs...),
                            Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = PIC_PDL ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(cudaStream_t s, dim3 grid, dim3 block, void (*kernel)(KArgs...), Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = PIC_PDL ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

// red-black Gauss-Seidel, one colour; thread (i2, j) of plane k = 1 + blockIdx.z
template <typename T>
__global__ void k_rbgs(T* __restrict__ u, const T* __restrict__ f, Dims d, T h2, int color, int zero)
{
    pdl_begin();
    const int i2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = 1 + blockIdx.z;
    if (i2 >= d.nx / 2 || j >= d.ny) return;
    const int i = 2 * i2 + ((j + k + color) & 1);
    const int P = d.nx * d.ny;
    const int n = k * P + j * d.nx + i;
    if (zero) {   // first sweep from a zero guess: the neighbours are still zero
        u[n] = (h2 * f[n]) * (T)(1.0 / 6.0);
        return;
    }
    const int row = n - i;
    const int ip = (i + 1 == d.nx) ? 0 : i + 1, im = (i == 0) ? d.nx - 1 : i - 1;
    const int jp = (j + 1 == d.ny) ? -j * d.nx : d.nx, jm = (j == 0) ? (d.ny - 1) * d.nx : -d.nx;
    const T s = u[row + ip] + u[row + im] + u[n + jp] + u[n + jm] + u[n + P] + u[n - P];
    u[n] = (s + h2 * f[n]) * (T)(1.0 / 6.0);
}

// The same half-sweep on a red-black split level (d.half > 0), by columns of
// node pairs.  Pair m = k * P/2 + j * nx/2 + i2 holds nodes 2 i2 and 2 i2 + 1
// of row (j, k), one of each colour, at m in the red half and m in the black
// half.  Every neighbour of the updated node (offset p = (j + k + colour) & 1
// in its pair) is of the other colour: in the same pair (x on one side), the
// pair next to it (x on the other side), pairs m -+ nx/2 (y) and m -+ P/2
// (z).  A thread walks its column up zp planes; the other colour's
// column values at k - 1, k, k + 1 roll through registers and the one at
// k + 2 is loaded a plane ahead.  Each node's sum is k_rbgs's, term by term.
constexpr int kRbPlanes = 16;   // most planes per block of the column kernels

// planes per block of a column kernel over `planes` planes: up to `most`, fewer
// when the columns alone would not give every SM four blocks
inline int column_planes(const Grid3& g, int planes, int most)
{
    const long long z = (long long)g.grid.x * g.grid.y * planes / (152LL * 4);
    return (int)std::max(1LL, std::min((long long)most, z));
}

template <typename T>
__global__ void k_rbgs_split(T* __restrict__ u, const T* __restrict__ f, Dims d, T h2, int color, int zero, int zp)
{
    pdl_begin();
    const int hx = d.nx >> 1, P2 = hx * d.ny;
    const int i2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = 1 + (int)blockIdx.z * zp;
    const int k1 = min(k0 + zp, d.nz);
    if (i2 >= hx || j >= d.ny || k0 >= k1) return;
    T* uc = u + (color ? d.half : 0);               // the colour being updated
    const T* fc = f + (color ? d.half : 0);
    const T* uo = u + (color ? 0 : d.half);         // the other colour
    int m = k0 * P2 + j * hx + i2;
    if (zero) {   // first sweep from a zero guess: the neighbours are still zero
        for (int k = k0; k < k1; ++k, m += P2) uc[m] = (h2 * fc[m]) * (T)(1.0 / 6.0);
        return;
    }
    const int dxp = (i2 + 1 == hx) ? 1 - hx : 1, dxm = (i2 == 0) ? hx - 1 : -1;
    const int dyp = (j + 1 == d.ny) ? -j * hx : hx, dym = (j == 0) ? (d.ny - 1) * hx : -hx;
    T om = uo[m - P2], oc = uo[m], op = uo[m + P2];
    for (int k = k0; k < k1; ++k, m += P2) {
        const T on = (k + 1 < k1) ? uo[m + 2 * P2] : op;
        const int p = (j + k + color) & 1;
        const T ox = uo[m + (p ? dxp : dxm)];
        const T xp = p ? ox : oc, xm = p ? oc : ox;
        const T s = xp + xm + uo[m + dyp] + uo[m + dym] + op + om;
        uc[m] = (s + h2 * fc[m]) * (T)(1.0 / 6.0);
        om = oc;
        oc = op;
        op = on;
    }
}

// k_rbgs_split with two adjacent pairs 2q, 2q + 1 per thread (nx a multiple of
// 4), so each load moves two values: the other colour's column values and f
// as one 8-byte (16-byte for double) load per plane, one scalar load for the x
// neighbour outside the two pairs.  The same sum per node, term by term.
template <typename T> struct Two;
template <> struct Two<float> { using V = float2; };
template <> struct Two<double> { using V = double2; };

template <typename T>
__global__ void k_rbgs_split2(T* __restrict__ u, const T* __restrict__ f, Dims d, T h2, int color, int zero, int zp)
{
    using V = typename Two<T>::V;
    pdl_begin();
    const int hx = d.nx >> 1, P2 = hx * d.ny, qx = hx >> 1;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = 1 + (int)blockIdx.z * zp;
    const int k1 = min(k0 + zp, d.nz);
    if (q >= qx || j >= d.ny || k0 >= k1) return;
    T* uc = u + (color ? d.half : 0);
    const T* fc = f + (color ? d.half : 0);
    const T* uo = u + (color ? 0 : d.half);
    int m = k0 * P2 + j * hx + 2 * q;   // even: 2-element aligned
    if (zero) {
        for (int k = k0; k < k1; ++k, m += P2) {
            const V ff = *reinterpret_cast<const V*>(fc + m);
            V r;
            r.x = (h2 * ff.x) * (T)(1.0 / 6.0);
            r.y = (h2 * ff.y) * (T)(1.0 / 6.0);
            *reinterpret_cast<V*>(uc + m) = r;
        }
        return;
    }
    const int dl = (q == 0) ? hx - 1 : -1;            // pair 2q - 1
    const int dr = (q + 1 == qx) ? 2 - hx : 2;        // pair 2q + 2
    const int dyp = (j + 1 == d.ny) ? -j * hx : hx, dym = (j == 0) ? (d.ny - 1) * hx : -hx;
    auto ld = [&](int at) { return *reinterpret_cast<const V*>(uo + at); };
    V om = ld(m - P2), oc = ld(m), op = ld(m + P2);
    for (int k = k0; k < k1; ++k, m += P2) {
        const V on = (k + 1 < k1) ? ld(m + 2 * P2) : op;
        const int p = (j + k + color) & 1;
        const T ox = uo[m + (p ? dr : dl)];
        const V yp = ld(m + dyp), ym = ld(m + dym);
        const V ff = *reinterpret_cast<const V*>(fc + m);
        const T xp0 = p ? oc.y : oc.x, xm0 = p ? oc.x : ox;
        const T xp1 = p ? ox : oc.y, xm1 = p ? oc.y : oc.x;
        const T s0 = xp0 + xm0 + yp.x + ym.x + op.x + om.x;
        const T s1 = xp1 + xm1 + yp.y + ym.y + op.y + om.y;
        V r;
        r.x = (s0 + h2 * ff.x) * (T)(1.0 / 6.0);
        r.y = (s1 + h2 * ff.y) * (T)(1.0 / 6.0);
        *reinterpret_cast<V*>(uc + m) = r;
        om = oc;
        oc = op;
        op = on;
    }
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

// residual f - A u at fine node (i, j, k)
template <typename T>
__device__ __forceinline__ T res_at(const T* __restrict__ u, const T* __restrict__ f, Dims d, int i, int j, int k,
                                    T inv_h2)
{
    const int P = d.nx * d.ny;
    const int ip = (i + 1 == d.nx) ? 0 : i + 1, im = (i == 0) ? d.nx - 1 : i - 1;
    const int jp = (j + 1 == d.ny) ? 0 : j + 1, jm = (j == 0) ? d.ny - 1 : j - 1;
    const int row = k * P + j * d.nx, n = row + i;
    const int c = (i + j + k) & 1, oc = c ^ 1;
    const T s = u[lix(d, row + ip, oc)] + u[lix(d, row + im, oc)] + u[lix(d, k * P + jp * d.nx + i, oc)] +
                u[lix(d, k * P + jm * d.nx + i, oc)] + u[lix(d, n + P, oc)] + u[lix(d, n - P, oc)];
    return f[lix(d, n, c)] - ((T)6 * u[lix(d, n, c)] - s) * inv_h2;
}

// Full-weighting restriction of the residual f - A u, computed on the fly.
// After the black half-sweep that ends the pre-smoothing the residual is zero
// at the black nodes, so only the 13 red points of the 27 enter (weight 1/8
// at the coincident node, 1/32 at the 12 with two odd offsets).  The coarse
// correction starts from zero: its first red half-sweep, h^2 f / 6 at the red
// coarse nodes, is written here as well.  Thread (I, J) of coarse plane
// K = 1 + blockIdx.z.
template <typename T>
__global__ void k_resid_restrict(const T* __restrict__ u, const T* __restrict__ f, T* __restrict__ fc,
                                 T* __restrict__ uc, Dims df, Dims dc, T inv_h2, T h2c)
{
    pdl_begin();
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = 1 + blockIdx.z;
    if (I >= dc.nx || J >= dc.ny) return;
    const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * K;
    const int im = (i0 == 0) ? df.nx - 1 : i0 - 1, ip = i0 + 1;
    const int jm = (j0 == 0) ? df.ny - 1 : j0 - 1, jp = j0 + 1;
    T e = res_at(u, f, df, im, jm, k0, inv_h2) + res_at(u, f, df, ip, jm, k0, inv_h2) +
          res_at(u, f, df, im, jp, k0, inv_h2) + res_at(u, f, df, ip, jp, k0, inv_h2);
    e += res_at(u, f, df, im, j0, k0 - 1, inv_h2) + res_at(u, f, df, ip, j0, k0 - 1, inv_h2) +
         res_at(u, f, df, im, j0, k0 + 1, inv_h2) + res_at(u, f, df, ip, j0, k0 + 1, inv_h2);
    e += res_at(u, f, df, i0, jm, k0 - 1, inv_h2) + res_at(u, f, df, i0, jp, k0 - 1, inv_h2) +
         res_at(u, f, df, i0, jm, k0 + 1, inv_h2) + res_at(u, f, df, i0, jp, k0 + 1, inv_h2);
    const T v = (T)0.125 * res_at(u, f, df, i0, j0, k0, inv_h2) + (T)0.03125 * e;
    const int nc = K * dc.nx * dc.ny + J * dc.nx + I;
    fc[nc] = v;
    if (((I + J + K) & 1) == 0) uc[nc] = h2c * v * (T)(1.0 / 6.0);
}

// trilinear interpolation of the coarse correction, added on the fine interior
template <typename T>
__global__ void k_prolong(T* __restrict__ uf, const T* __restrict__ uc, Dims df, Dims dc)
{
    pdl_begin();
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
    uf[lix(df, k * df.nx * df.ny + j * df.nx + i, (i + j + k) & 1)] += v;
}

// The same interpolation, one thread per coarse cell (I, J, K): its 8 corner
// values are loaded once and give the 2 x 2 x 2 fine nodes (2I + a, 2J + b,
// 2K + c), each summed exactly as in k_prolong (a coincident axis repeats its
// corner), so the result is bit-identical with 8 times fewer coarse loads.
template <typename T>
__global__ void k_prolong_cell(T* __restrict__ uf, const T* __restrict__ uc, Dims df, Dims dc)
{
    pdl_begin();
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = blockIdx.z;
    if (I >= dc.nx || J >= dc.ny) return;
    const int I1 = (I + 1 == dc.nx) ? 0 : I + 1, J1 = (J + 1 == dc.ny) ? 0 : J + 1;
    const int Pc = dc.nx * dc.ny;
    const T* a0 = uc + K * Pc;
    const T* a1 = a0 + Pc;
    // c[z][y][x]: corners at (I or I1, J or J1, K or K + 1)
    const T c000 = a0[J * dc.nx + I], c001 = a0[J * dc.nx + I1], c010 = a0[J1 * dc.nx + I], c011 = a0[J1 * dc.nx + I1];
    const T c100 = a1[J * dc.nx + I], c101 = a1[J * dc.nx + I1], c110 = a1[J1 * dc.nx + I], c111 = a1[J1 * dc.nx + I1];
    const int P = df.nx * df.ny;
#pragma unroll
    for (int cz = 0; cz < 2; ++cz) {
        const int k = 2 * K + cz;
        if (k < 1 || k > df.nz - 1) continue;
        // K1 = K + cz: the second plane term repeats the first when cz = 0
        const T z0[4] = {c000, c001, c010, c011};
        const T z1[4] = {cz ? c100 : c000, cz ? c101 : c001, cz ? c110 : c010, cz ? c111 : c011};
#pragma unroll
        for (int by = 0; by < 2; ++by) {
            const int j = 2 * J + by;
#pragma unroll
            for (int bx = 0; bx < 2; ++bx) {
                const int i = 2 * I + bx;
                // terms in k_prolong's order: a0[J0 I0], a0[J0 I1], a0[J1 I0], a0[J1 I1], then a1 likewise,
                // with I1 = I0 and J1 = J0 on the even axes
                const T p00 = z0[0], p01 = z0[bx ? 1 : 0], p10 = z0[by ? 2 : 0], p11 = z0[(by ? 2 : 0) + (bx ? 1 : 0)];
                const T q00 = z1[0], q01 = z1[bx ? 1 : 0], q10 = z1[by ? 2 : 0], q11 = z1[(by ? 2 : 0) + (bx ? 1 : 0)];
                const T v = (T)0.125 * (p00 + p01 + p10 + p11 + q00 + q01 + q10 + q11);
                uf[lix(df, k * P + j * df.nx + i, (i + j + k) & 1)] += v;
            }
        }
    }
}

// ---- red-black split finest level: restriction and prolongation by columns --
constexpr int kSplitPlanes = 8;   // most coarse planes per block of the prolongation below

// Red residual r = f - A u at the red nodes of a split level (the black ones
// are zero after the black half-sweep), written to rr[m] at the red node's
// pair index; columns of node pairs as in k_rbgs_split, the same terms in
// res_at's order.
template <typename T>
__global__ void k_resid_red_split(const T* __restrict__ u, const T* __restrict__ f, T* __restrict__ rr, Dims d,
                                  T inv_h2, int zp)
{
    pdl_begin();
    const int hx = d.nx >> 1, P2 = hx * d.ny;
    const int i2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = 1 + (int)blockIdx.z * zp;
    const int k1 = min(k0 + zp, d.nz);
    if (i2 >= hx || j >= d.ny || k0 >= k1) return;
    const T* ur = u;               // red
    const T* ub = u + d.half;      // black: every neighbour of a red node
    const int dxp = (i2 + 1 == hx) ? 1 - hx : 1, dxm = (i2 == 0) ? hx - 1 : -1;
    const int dyp = (j + 1 == d.ny) ? -j * hx : hx, dym = (j == 0) ? (d.ny - 1) * hx : -hx;
    int m = k0 * P2 + j * hx + i2;
    T om = ub[m - P2], oc = ub[m], op = ub[m + P2];
    for (int k = k0; k < k1; ++k, m += P2) {
        const T on = (k + 1 < k1) ? ub[m + 2 * P2] : op;
        const int p = (j + k) & 1;   // offset of the red node in its pair
        const T ox = ub[m + (p ? dxp : dxm)];
        const T xp = p ? ox : oc, xm = p ? oc : ox;
        const T s = xp + xm + ub[m + dyp] + ub[m + dym] + op + om;
        rr[m] = f[m] - ((T)6 * ur[m] - s) * inv_h2;
        om = oc;
        oc = op;
        op = on;
    }
}

// k_resid_red_split with two adjacent pairs per thread (as k_rbgs_split2)
template <typename T>
__global__ void k_resid_red_split2(const T* __restrict__ u, const T* __restrict__ f, T* __restrict__ rr, Dims d,
                                   T inv_h2, int zp)
{
    using V = typename Two<T>::V;
    pdl_begin();
    const int hx = d.nx >> 1, P2 = hx * d.ny, qx = hx >> 1;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = 1 + (int)blockIdx.z * zp;
    const int k1 = min(k0 + zp, d.nz);
    if (q >= qx || j >= d.ny || k0 >= k1) return;
    const T* ur = u;
    const T* ub = u + d.half;
    const int dl = (q == 0) ? hx - 1 : -1, dr = (q + 1 == qx) ? 2 - hx : 2;
    const int dyp = (j + 1 == d.ny) ? -j * hx : hx, dym = (j == 0) ? (d.ny - 1) * hx : -hx;
    int m = k0 * P2 + j * hx + 2 * q;
    auto ld = [&](const T* a, int at) { return *reinterpret_cast<const V*>(a + at); };
    V om = ld(ub, m - P2), oc = ld(ub, m), op = ld(ub, m + P2);
    for (int k = k0; k < k1; ++k, m += P2) {
        const V on = (k + 1 < k1) ? ld(ub, m + 2 * P2) : op;
        const int p = (j + k) & 1;   // offset of the red nodes in their pairs
        const T ox = ub[m + (p ? dr : dl)];
        const V yp = ld(ub, m + dyp), ym = ld(ub, m + dym), uu = ld(ur, m), ff = ld(f, m);
        const T xp0 = p ? oc.y : oc.x, xm0 = p ? oc.x : ox;
        const T xp1 = p ? ox : oc.y, xm1 = p ? oc.y : oc.x;
        const T s0 = xp0 + xm0 + yp.x + ym.x + op.x + om.x;
        const T s1 = xp1 + xm1 + yp.y + ym.y + op.y + om.y;
        V r;
        r.x = ff.x - ((T)6 * uu.x - s0) * inv_h2;
        r.y = ff.y - ((T)6 * uu.y - s1) * inv_h2;
        *reinterpret_cast<V*>(rr + m) = r;
        om = oc;
        oc = op;
        op = on;
    }
}

// Full-weighting restriction of the red residuals rr (as k_resid_restrict:
// 1/8 at the coincident node, 1/32 at the 12 with two odd offsets, in its
// order of terms), and the coarse level's first red half-sweep from zero.
template <typename T>
__global__ void k_restrict_red(const T* __restrict__ rr, T* __restrict__ fc, T* __restrict__ uc, Dims df, Dims dc,
                               T h2c)
{
    pdl_begin();
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int K = 1 + blockIdx.z;
    if (I >= dc.nx || J >= dc.ny) return;
    const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * K;
    const int im = (i0 == 0) ? df.nx - 1 : i0 - 1, ip = i0 + 1;
    const int jm = (j0 == 0) ? df.ny - 1 : j0 - 1, jp = j0 + 1;
    const int P = df.nx * df.ny;
    auto r = [&](int i, int j, int k) { return rr[(k * P + j * df.nx + i) >> 1]; };
    T e = r(im, jm, k0) + r(ip, jm, k0) + r(im, jp, k0) + r(ip, jp, k0);
    e += r(im, j0, k0 - 1) + r(ip, j0, k0 - 1) + r(im, j0, k0 + 1) + r(ip, j0, k0 + 1);
    e += r(i0, jm, k0 - 1) + r(i0, jp, k0 - 1) + r(i0, jm, k0 + 1) + r(i0, jp, k0 + 1);
    const T v = (T)0.125 * r(i0, j0, k0) + (T)0.03125 * e;
    const int nc = K * dc.nx * dc.ny + J * dc.nx + I;
    const int col = (I + J + K) & 1;
    fc[lix(dc, nc, col)] = v;
    if (col == 0) uc[lix(dc, nc, 0)] = h2c * v * (T)(1.0 / 6.0);
}

// k_prolong_cell onto a split level: thread (I, J) walks zp coarse
// planes of its column, the corners of plane K + 1 reused as those of the
// next cell's plane K; the fine pair (I, 2J + b, 2K + c) gets its two nodes'
// values added at pair index m in the red and black halves.
template <typename T>
__global__ void k_prolong_split(T* __restrict__ uf, const T* __restrict__ uc, Dims df, Dims dc, int zp)
{
    pdl_begin();
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y * blockDim.y + threadIdx.y;
    const int Kb = (int)blockIdx.z * zp;
    const int Ke = min(Kb + zp, dc.nz);
    if (I >= dc.nx || J >= dc.ny || Kb >= Ke) return;
    const int I1 = (I + 1 == dc.nx) ? 0 : I + 1, J1 = (J + 1 == dc.ny) ? 0 : J + 1;
    const int Pc = dc.nx * dc.ny, hx = df.nx >> 1, P2 = hx * df.ny;
    // a corner of coarse plane K (the coarse level may itself be split)
    auto cr = [&](int K, int i, int j) { return uc[lix(dc, K * Pc + j * dc.nx + i, (i + j + K) & 1)]; };
    T c000 = cr(Kb, I, J), c001 = cr(Kb, I1, J), c010 = cr(Kb, I, J1), c011 = cr(Kb, I1, J1);
    for (int K = Kb; K < Ke; ++K) {
        const T c100 = cr(K + 1, I, J), c101 = cr(K + 1, I1, J), c110 = cr(K + 1, I, J1), c111 = cr(K + 1, I1, J1);
        // the 8 fine values of this cell: addresses and old values first (all
        // loads in flight together), then the sums and stores
        int adr[2][2][2];
        T old[2][2][2];
#pragma unroll
        for (int cz = 0; cz < 2; ++cz)
#pragma unroll
            for (int by = 0; by < 2; ++by) {
                const int k = 2 * K + cz, j = 2 * J + by;
                const int m = k * P2 + j * hx + I;
                const int c0 = (j + k) & 1;   // colour of node 0 of the pair
                adr[cz][by][0] = (c0 ? df.half : 0) + m;
                adr[cz][by][1] = (c0 ? 0 : df.half) + m;
                const bool in = k >= 1 && k <= df.nz - 1;
#pragma unroll
                for (int bx = 0; bx < 2; ++bx) old[cz][by][bx] = in ? uf[adr[cz][by][bx]] : (T)0;
            }
#pragma unroll
        for (int cz = 0; cz < 2; ++cz) {
            const int k = 2 * K + cz;
            if (k < 1 || k > df.nz - 1) continue;
            const T z0[4] = {c000, c001, c010, c011};
            const T z1[4] = {cz ? c100 : c000, cz ? c101 : c001, cz ? c110 : c010, cz ? c111 : c011};
#pragma unroll
            for (int by = 0; by < 2; ++by)
#pragma unroll
                for (int bx = 0; bx < 2; ++bx) {
                    const T p00 = z0[0], p01 = z0[bx ? 1 : 0], p10 = z0[by ? 2 : 0], p11 = z0[(by ? 2 : 0) + (bx ? 1 : 0)];
                    const T q00 = z1[0], q01 = z1[bx ? 1 : 0], q10 = z1[by ? 2 : 0], q11 = z1[(by ? 2 : 0) + (bx ? 1 : 0)];
                    const T v = (T)0.125 * (p00 + p01 + p10 + p11 + q00 + q01 + q10 + q11);
                    uf[adr[cz][by][bx]] = old[cz][by][bx] + v;
                }
        }
        c000 = c100;
        c001 = c101;
        c010 = c110;
        c011 = c111;
    }
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
            const int col = (i + j + k) & 1;
            double c = phi[n];
            double s = 0.0;
            if (e) {
                c += (double)e[lix(d, n, col)];
#pragma unroll
                for (int q = 0; q < 6; ++q) s += phi[nb[q]] + (double)e[lix(d, nb[q], col ^ 1)];
            } else {
#pragma unroll
                for (int q = 0; q < 6; ++q) s += phi[nb[q]];
            }
            if (phi_out) phi_out[n] = c;
            const double res = f[n] - (6.0 * c - s) * inv_h2;
            r[lix(d, n, col)] = (T)res;
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
    const int k = 1 + (int)blockIdx.z;
    const int n = (k * d.ny + j) * d.nx + i;
    phi[n] += (double)e[lix(d, n, (i + j + k) & 1)];
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

// ---- the levels below the grid-wide ones: one thread-block cluster ---------
// Every level from mg_tail down is held in the shared memory of the CTAs of
// one cluster.  A level is cut into z slabs, one per CTA (slab boundaries
// nested between levels: fine plane 2K and coarse plane K have the same
// owner); the smallest levels sit in CTA 0 alone.  Neighbour planes owned by
// another CTA are read through distributed shared memory, and the phases of
// the V-cycle are separated by cluster barriers (CTA barriers on the levels
// of CTA 0 alone).  The coarsest level is solved with the dense inverse or by
// many red-black sweeps.
constexpr int kTailMax = 8;
constexpr int kClThreads = PIC_MG_CL_THREADS;

// n / d for 0 <= n < 2^31 by a multiply-high and a shift (Granlund and
// Montgomery's division by invariant integers, round-up variant)
struct FastDiv {
    unsigned int m;
    int s;
};
inline FastDiv fast_div(int d)
{
    int l = 0;
    while ((1u << l) < (unsigned)d) ++l;
    const unsigned long long m = ((1ull << 32) * ((1ull << l) - (unsigned long long)d)) / (unsigned long long)d + 1;
    return FastDiv{(unsigned int)m, l};
}
__device__ __forceinline__ int fdiv(int n, FastDiv f)
{
    return (int)((__umulhi((unsigned)n, f.m) + (unsigned)n) >> f.s);
}

template <typename T>
struct ClusterLevels {
    int n;                            // levels; index 0 is mg_tail, n - 1 the coarsest
    int single;                       // first level held by CTA 0 alone (<= n - 1)
    int nx[kTailMax], ny[kTailMax], nz[kTailMax];
    T h2[kTailMax], ih2[kTailMax];
    FastDiv f_hx[kTailMax], f_ph[kTailMax];   // nx / 2 and nx ny / 2
    FastDiv f_x[kTailMax], f_p[kTailMax];     // nx and nx ny
    unsigned int off[kTailMax];       // byte offset of the level's u block (its f block follows)
    int mp[kTailMax];                 // planes reserved per CTA
    int pbase[kTailMax];              // first entry of the level in the plane pointer tables
    unsigned int ptr_off;             // byte offset of the tables (u pointers, then f pointers)
    int nplanes;                      // entries per table
    T* gu;                            // correction of level 0 (out, interior planes)
    const T* gf;                      // right-hand side of level 0 (in)
    const T* ainv;                    // dense inverse of the coarsest operator, or null
    int sweeps;                       // coarsest-level sweeps without an inverse
};

// first plane owned by CTA r of C on a distributed level with planes 0..nz (r = C gives nz + 1)
__device__ __forceinline__ int cl_kfirst(int r, int C, int nz)
{
    if (r >= C) return nz + 1;
    return (r * nz + C - 1) / C;
}
__device__ __forceinline__ int cl_owner(int k, int C, int nz)
{
    const int o = (k * C) / nz;
    return o < C - 1 ? o : C - 1;
}
// planes [k0, k1) that CTA r holds: its slab, or all of a level every CTA holds
__device__ __forceinline__ void cl_planes(int r, int C, int nz, bool single, int& k0, int& k1)
{
    if (single) {
        k0 = 0;
        k1 = nz + 1;
    } else {
        k0 = cl_kfirst(r, C, nz);
        k1 = cl_kfirst(r + 1, C, nz);
    }
}

template <typename T>
struct ClView {
    T* const* pu;     // plane pointers (generic addresses, local or in another CTA)
    T* const* pf;
    int r, C;
};

// one level as this CTA sees it: levels held by CTA 0 alone are addressed in
// its own shared memory (plane k at u + k P), distributed levels through the
// plane tables
template <typename T>
struct Lv {
    T* const* pu;
    T* const* pf;
    T* u;
    T* f;
    int nx, ny, nz, P;
    bool local;
    __device__ __forceinline__ T* U(int k) const { return local ? u + k * P : pu[k]; }
    __device__ __forceinline__ T* F(int k) const { return local ? f + k * P : pf[k]; }
};

// One colour of red-black Gauss-Seidel on the interior planes [klo, khi]
// (omega = 1: a node's new value does not depend on its old one).  Each
// thread keeps one half-column (i2, j) of a plane and walks the planes
// k = klo + g, klo + g + G, ...; the node of the colour in plane k is
// i = 2 i2 or 2 i2 + 1 by the parity of j + k.
template <typename T>
__device__ __forceinline__ void cl_rbgs(const Lv<T> a, T h2, int klo, int khi, int color, FastDiv f_ph, FastDiv f_hx)
{
    if (khi < klo) return;
    const int bd = blockDim.x, t = threadIdx.x;
    const int hx = a.nx / 2, ph = hx * a.ny;
    int g = 0, G = 1, c = t, cstep = bd;
    if (ph <= bd) {
        g = fdiv(t, f_ph);
        G = bd / ph;
        if (g >= G) return;
        c = t - g * ph;
        cstep = ph;
    }
    for (; c < ph; c += cstep) {
        const int j = fdiv(c, f_hx), i2 = c - j * hx;
        const int jr = j * a.nx;
        const int jpr = (j + 1 == a.ny ? 0 : j + 1) * a.nx, jmr = (j == 0 ? a.ny - 1 : j - 1) * a.nx;
        const int e0 = 2 * i2, e1 = e0 + 1;
        const int em0 = (i2 == 0) ? a.nx - 1 : e0 - 1;
        const int ep1 = (e1 + 1 == a.nx) ? 0 : e1 + 1;
        for (int k = klo + g; k <= khi; k += G) {
            const bool odd = ((j + k + color) & 1) != 0;
            const int i = odd ? e1 : e0, im = odd ? e0 : em0, ip = odd ? ep1 : e1;
            T* u = a.U(k);
            const int n = jr + i;
            const T s = u[jr + im] + u[jr + ip] + u[jpr + i] + u[jmr + i] + a.U(k + 1)[n] + a.U(k - 1)[n];
            u[n] = (s + h2 * a.F(k)[n]) * (T)(1.0 / 6.0);
        }
    }
}

// residual f - A u at node (i, j) of plane k
template <typename T>
__device__ __forceinline__ T cl_res(const Lv<T> a, T ih2, int i, int j, int k)
{
    const T* u = a.U(k);
    const int ip = (i + 1 == a.nx) ? 0 : i + 1, im = (i == 0) ? a.nx - 1 : i - 1;
    const int jp = (j + 1 == a.ny) ? 0 : j + 1, jm = (j == 0) ? a.ny - 1 : j - 1;
    const int n = j * a.nx + i;
    const T s = u[j * a.nx + ip] + u[j * a.nx + im] + u[jp * a.nx + i] + u[jm * a.nx + i] + a.U(k + 1)[n] +
                a.U(k - 1)[n];
    return a.F(k)[n] - ((T)6 * u[n] - s) * ih2;
}

// Full-weighting restriction of the fine residual to the coarse interior
// planes [Klo, Khi].  After a black half-sweep the residual is zero at the
// black nodes, so only the 13 red points of the 27 enter: weight 1/8 at the
// coincident node and 1/32 at the 12 with two odd offsets.  The coarse
// correction starts from zero, so its first red half-sweep (h^2 f / 6) is
// written here too.  With bcast > 0 the coarse level is one that every CTA
// holds, and the values go to all bcast copies.
template <typename T>
__device__ __forceinline__ void cl_restrict(const Lv<T> a, const Lv<T> b, T ih2, T h2c, int Klo, int Khi, FastDiv f_pc,
                            FastDiv f_xc, int bcast)
{
    if (Khi < Klo) return;
    const int pc = b.nx * b.ny;
    const int total = (Khi - Klo + 1) * pc;
    for (int m = threadIdx.x; m < total; m += blockDim.x) {
        const int kk = fdiv(m, f_pc);
        const int rem = m - kk * pc;
        const int J = fdiv(rem, f_xc);
        const int I = rem - J * b.nx;
        const int K = Klo + kk;
        const int i0 = 2 * I, j0 = 2 * J, k0 = 2 * K;
        const int im = (i0 == 0) ? a.nx - 1 : i0 - 1, ip = i0 + 1;
        const int jm = (j0 == 0) ? a.ny - 1 : j0 - 1, jp = j0 + 1;
        T e = cl_res(a, ih2, im, jm, k0) + cl_res(a, ih2, ip, jm, k0) + cl_res(a, ih2, im, jp, k0) +
              cl_res(a, ih2, ip, jp, k0);
        e += cl_res(a, ih2, im, j0, k0 - 1) + cl_res(a, ih2, ip, j0, k0 - 1) + cl_res(a, ih2, im, j0, k0 + 1) +
             cl_res(a, ih2, ip, j0, k0 + 1);
        e += cl_res(a, ih2, i0, jm, k0 - 1) + cl_res(a, ih2, i0, jp, k0 - 1) + cl_res(a, ih2, i0, jm, k0 + 1) +
             cl_res(a, ih2, i0, jp, k0 + 1);
        const T fc = (T)0.125 * cl_res(a, ih2, i0, j0, k0) + (T)0.03125 * e;
        const int nc = J * b.nx + I;
        const bool red = ((I + J + K) & 1) == 0;
        const T uc = h2c * fc * (T)(1.0 / 6.0);
        if (bcast == 0) {
            b.F(K)[nc] = fc;
            if (red) b.U(K)[nc] = uc;
        } else {
            cg::cluster_group cl = cg::this_cluster();
            for (int q = 0; q < bcast; ++q) {
                *cl.map_shared_rank(b.F(K) + nc, q) = fc;
                if (red) *cl.map_shared_rank(b.U(K) + nc, q) = uc;
            }
        }
    }
}

// trilinear interpolation of the coarse correction added on the fine interior
// planes [klo, khi]; threads keep a column (i, j) as in cl_rbgs
template <typename T>
__device__ __forceinline__ void cl_prolong(const Lv<T> a, const Lv<T> b, int klo, int khi, FastDiv f_p, FastDiv f_x)
{
    if (khi < klo) return;
    const int bd = blockDim.x, t = threadIdx.x;
    int g = 0, G = 1, c = t, cstep = bd;
    if (a.P <= bd) {
        g = fdiv(t, f_p);
        G = bd / a.P;
        if (g >= G) return;
        c = t - g * a.P;
        cstep = a.P;
    }
    for (; c < a.P; c += cstep) {
        const int j = fdiv(c, f_x), i = c - j * a.nx;
        const int I0 = i >> 1, I1 = (i & 1) ? ((I0 + 1 == b.nx) ? 0 : I0 + 1) : I0;
        const int J0 = j >> 1, J1 = (j & 1) ? ((J0 + 1 == b.ny) ? 0 : J0 + 1) : J0;
        const int o00 = J0 * b.nx + I0, o01 = J0 * b.nx + I1, o10 = J1 * b.nx + I0, o11 = J1 * b.nx + I1;
        for (int k = klo + g; k <= khi; k += G) {
            const int K0 = k >> 1, K1 = K0 + (k & 1);
            const T* a0 = b.U(K0);
            const T* a1 = b.U(K1);
            // a coincident axis repeats its node, so the 1/8 weights give 1/2 or 1 per axis
            const T v = (T)0.125 * (a0[o00] + a0[o01] + a0[o10] + a0[o11] + a1[o00] + a1[o01] + a1[o10] + a1[o11]);
            a.U(k)[c] += v;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kClThreads) k_vcycle_cluster(const ClusterLevels<T> Lp)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    extern __shared__ __align__(16) unsigned char smem[];
    // the level table is indexed by level at run time: keep it in shared memory
    __shared__ ClusterLevels<T> L;
    if (threadIdx.x == 0) L = Lp;
    __syncthreads();
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank(), C = (int)cl.num_blocks();
    T** pu = reinterpret_cast<T**>(smem + L.ptr_off);
    T** pf = pu + L.nplanes;
    // plane tables of the distributed levels: every plane, wherever it is held
    for (int e = threadIdx.x; e < L.nplanes; e += blockDim.x) {
        int l = 0;
        while (l + 1 < L.n && e >= L.pbase[l + 1]) ++l;
        const int k = e - L.pbase[l];
        const bool sg = l >= L.single;
        const int o = sg ? r : cl_owner(k, C, L.nz[l]);
        const int P = L.nx[l] * L.ny[l];
        T* lu = reinterpret_cast<T*>(smem + L.off[l]) + (size_t)(k - (sg ? 0 : cl_kfirst(o, C, L.nz[l]))) * P;
        T* lf = lu + (size_t)L.mp[l] * P;
        pu[e] = cl.map_shared_rank(lu, o);
        pf[e] = cl.map_shared_rank(lf, o);
    }
    // this CTA's planes start at zero (the electrode planes of the corrections stay zero)
    for (int l = 0; l < L.n; ++l) {
        T* b = reinterpret_cast<T*>(smem + L.off[l]);
        const int words = 2 * L.mp[l] * L.nx[l] * L.ny[l];
        for (int t = threadIdx.x; t < words; t += blockDim.x) b[t] = (T)0;
    }
    __syncthreads();
    auto lv = [&](int l) {
        Lv<T> a;
        a.pu = pu + L.pbase[l];
        a.pf = pf + L.pbase[l];
        a.u = reinterpret_cast<T*>(smem + L.off[l]);
        a.nx = L.nx[l];
        a.ny = L.ny[l];
        a.nz = L.nz[l];
        a.P = a.nx * a.ny;
        a.f = a.u + (size_t)L.mp[l] * a.P;
        a.local = l >= L.single;
        return a;
    };
    auto range = [&](int l, int& klo, int& khi) {
        int k0, k1;
        cl_planes(r, C, L.nz[l], l >= L.single, k0, k1);
        klo = max(1, k0);
        khi = min(L.nz[l] - 1, k1 - 1);
    };
    auto sync_level = [&](int l) {
        if (l < L.single) cl.sync();
        else __syncthreads();
    };
    {   // right-hand side of the first level on this CTA's planes, and the first
        // red half-sweep from a zero guess (h^2 f / 6 at the red interior nodes)
        const Lv<T> a = lv(0);
        int k0, k1;
        cl_planes(r, C, a.nz, 0 >= L.single, k0, k1);
        const T h6 = L.h2[0] * (T)(1.0 / 6.0);
        for (int k = k0; k < k1; ++k) {
            T* fk = a.F(k);
            T* uk = a.U(k);
            for (int t = threadIdx.x; t < a.P; t += blockDim.x) {
                const T v = L.gf[(size_t)k * a.P + t];
                fk[t] = v;
                const int j = fdiv(t, L.f_x[0]);
                if (k > 0 && k < a.nz && ((t - j * a.nx + j + k) & 1) == 0) uk[t] = h6 * v;
            }
        }
    }
    cl.sync();
    // down: black, red, black half-sweeps (the first red one is done), residual
    // restricted to the next level with that level's first red half-sweep
    for (int l = 0; l + 1 < L.n; ++l) {
        const Lv<T> a = lv(l);
        int klo, khi;
        range(l, klo, khi);
        cl_rbgs(a, L.h2[l], klo, khi, 1, L.f_ph[l], L.f_hx[l]);
        sync_level(l);
        cl_rbgs(a, L.h2[l], klo, khi, 0, L.f_ph[l], L.f_hx[l]);
        sync_level(l);
        cl_rbgs(a, L.h2[l], klo, khi, 1, L.f_ph[l], L.f_hx[l]);
        sync_level(l);
        {   // coarse planes K whose fine plane 2K this CTA holds
            int f0, f1;
            cl_planes(r, C, a.nz, l >= L.single, f0, f1);
            const int Klo = max(1, (f0 + 1) / 2), Khi = min(L.nz[l + 1] - 1, (f1 - 1) / 2);
            const int bcast = (l < L.single && l + 1 >= L.single) ? C : 0;
            cl_restrict(a, lv(l + 1), L.ih2[l], L.h2[l + 1], Klo, Khi, L.f_p[l + 1], L.f_x[l + 1], bcast);
        }
        sync_level(l);
    }
    {   // the coarsest level (held by every CTA, solved by each)
        const int c = L.n - 1;
        const Lv<T> a = lv(c);
        const int nun = a.P * (a.nz - 1);
        if (L.ainv) {
            for (int m = threadIdx.x; m < nun; m += blockDim.x) {
                const T* row = L.ainv + (size_t)m * nun;
                T acc = (T)0;
                for (int q = 0; q < nun; ++q) acc += row[q] * a.f[a.P + q];
                a.u[a.P + m] = acc;
            }
            __syncthreads();
        } else {
            for (int s = 0; s < L.sweeps; ++s) {
                cl_rbgs(a, L.h2[c], 1, a.nz - 1, s == 0 ? 1 : 0, L.f_ph[c], L.f_hx[c]);
                __syncthreads();
                cl_rbgs(a, L.h2[c], 1, a.nz - 1, s == 0 ? 0 : 1, L.f_ph[c], L.f_hx[c]);
                __syncthreads();
            }
        }
    }
    // up: prolongation and four half-sweeps
    for (int l = L.n - 2; l >= 0; --l) {
        const Lv<T> a = lv(l);
        int klo, khi;
        range(l, klo, khi);
        cl_prolong(a, lv(l + 1), klo, khi, L.f_p[l], L.f_x[l]);
        sync_level(l);
        for (int h = 0; h < 4; ++h) {
            cl_rbgs(a, L.h2[l], klo, khi, h & 1, L.f_ph[l], L.f_hx[l]);
            sync_level(l);
        }
    }
    {   // the first level's correction back to global memory
        if (0 >= L.single && r != 0) return;
        const Lv<T> a = lv(0);
        int klo, khi;
        range(0, klo, khi);
        for (int k = klo; k <= khi; ++k) {
            const T* uk = a.U(k);
            for (int t = threadIdx.x; t < a.P; t += blockDim.x) L.gu[(size_t)k * a.P + t] = uk[t];
        }
    }
}

constexpr size_t kClSmemMax = 220 * 1024;

// layout of the levels l0.. for a cluster of C CTAs; false if it does not fit
template <typename T>
bool cluster_levels(const pic_ctx* c, int l0, int C, ClusterLevels<T>* out, size_t* smem)
{
    ClusterLevels<T> L{};
    L.n = (int)c->mg.size() - l0;
    if (L.n < 1 || L.n > kTailMax) return false;
    L.single = L.n - 1;
    for (int q = 0; q < L.n; ++q)
        if (C == 1 || c->mg[l0 + q].nodes <= kTailNodes) {
            L.single = q;
            break;
        }
    size_t off = 0;
    int pb = 0;
    for (int q = 0; q < L.n; ++q) {
        const MGLevel& M = c->mg[l0 + q];
        L.nx[q] = M.nx;
        L.ny[q] = M.ny;
        L.nz[q] = M.nz;
        L.h2[q] = (T)(M.h * M.h);
        L.ih2[q] = (T)(1.0 / (M.h * M.h));
        L.f_hx[q] = fast_div(M.nx / 2);
        L.f_ph[q] = fast_div(M.nx * M.ny / 2);
        L.f_x[q] = fast_div(M.nx);
        L.f_p[q] = fast_div(M.nx * M.ny);
        L.mp[q] = q >= L.single ? M.nz + 1 : (M.nz + C - 1) / C + 1;
        L.off[q] = (unsigned int)off;
        off += (2 * sizeof(T) * (size_t)L.mp[q] * M.nx * M.ny + 15) / 16 * 16;
        L.pbase[q] = pb;
        pb += M.nz + 1;
    }
    L.ptr_off = (unsigned int)off;
    L.nplanes = pb;
    off += 2 * sizeof(T*) * (size_t)pb;
    L.gu = (T*)c->mg[l0].u;
    L.gf = (const T*)c->mg[l0].f;
    L.ainv = (const T*)c->coarse_inv;
    const MGLevel& Cl = c->mg.back();
    const int m = std::max(std::max(Cl.nx, Cl.ny), Cl.nz);
    L.sweeps = std::min(4 * m * m + 16, 2000);
    if (off > kClSmemMax) return false;
    if (out) *out = L;
    if (smem) *smem = off;
    return true;
}

template <typename T>
cudaError_t launch_cluster(cudaStream_t s, const ClusterLevels<T>& L, int C, size_t smem, bool query, int* fits)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)C, 1, 1);
    cfg.blockDim = dim3(kClThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (query) {
        cudaError_t e = cudaFuncSetAttribute(k_vcycle_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kClSmemMax);
        if (e == cudaSuccess && C > 8)
            e = cudaFuncSetAttribute(k_vcycle_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        int n = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, k_vcycle_cluster<T>, &cfg);
        *fits = e == cudaSuccess && n > 0;
        cudaGetLastError();
        return cudaSuccess;
    }
    return cudaLaunchKernelEx(&cfg, k_vcycle_cluster<T>, L);
}

// ---- exact solve of one coarse level in one thread-block cluster -----------
// The rediscretised operator (6 u - neighbour sum) / h^2 with periodic x, y
// and zero Dirichlet planes separates: an orthonormal real Fourier basis
// (constant, cos/sin pairs, alternating) diagonalises the periodic second
// differences in x and y with eigenvalues 2 - 2 cos(2 pi p / n), and each
// resulting mode (mx, my) leaves a constant-coefficient tridiagonal system in z,
//     (2 + lx + ly) v_k - v_(k-1) - v_(k+1) = h^2 fhat_k,  v_0 = v_nz = 0,
// solved by the Thomas recurrence with pivots p_k = 1 / (d - p_(k-1))
// precomputed per mode.  CTA r of C holds a z slab of planes (transforms in
// x and y are local) and a block of modes (the z solves are local); the
// spectral values move between the two layouts through distributed shared
// memory.
template <typename T>
struct ExactLevel {
    int nx, ny, nz;
    int rp;              // row pitch of the plane buffers in shared memory (nx + 4)
    T h2;
    const T* Q;          // Qx, Qx transposed, Qy, Qy transposed; rows of Qx, Qy are basis vectors
    const T* p;          // Thomas pivots, (nz - 1) per mode, mode m = my nx + mx
    const T* gf;         // right-hand side of the level (in)
    T* gu;               // correction of the level (out, interior planes)
    int mp;              // planes reserved per CTA
    int mm;              // modes per CTA
    unsigned int off_a, off_b, off_g, off_p;   // byte offsets in shared memory (Q at 0)
    FastDiv f_x, f_n, f_x4, f_y4, f_t2;        // nx, nz - 1, nx / 4, ny / 4, (ny / 4)(nx / 4)
};

// four consecutive values (16-byte aligned)
__device__ __forceinline__ void ld4(const float* p, float v[4])
{
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4])
{
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float v[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double v[4])
{
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}

// Out[r][c] = scale * sum_s X(r, s) Y(s, c) on one 4 x 4 tile, with X read
// as four rows (one value each per s, rows xp apart) or as a 4-vector per s,
// and Y as a 4-vector per s.
template <typename T, bool XVEC>
__device__ __forceinline__ void tile4(const T* x, int xs, int xp, const T* y, int ys, int n, T acc[4][4])
{
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
#pragma unroll 4
    for (int s = 0; s < n; ++s) {
        T xv[4], yv[4];
        if (XVEC) {
            ld4(x + s * xs, xv);
        } else {
#pragma unroll
            for (int a = 0; a < 4; ++a) xv[a] = x[a * xp + s * xs];
        }
        ld4(y + s * ys, yv);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += xv[a] * yv[b];
    }
}

template <typename T>
__global__ void __launch_bounds__(kClThreads) k_coarse_exact(const ExactLevel<T> E)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank(), C = (int)cl.num_blocks();
    const int nx = E.nx, ny = E.ny, nz = E.nz, P = nx * ny, N = nz - 1, rp = E.rp, pp = ny * E.rp;
    const int bd = blockDim.x, t = threadIdx.x;
    T* Qx = reinterpret_cast<T*>(smem);   // [m][i]
    T* QxT = Qx + nx * nx;                // [i][m]
    T* Qy = QxT + nx * nx;                // [m][j]
    T* QyT = Qy + ny * ny;                // [j][m]
    T* A = reinterpret_cast<T*>(smem + E.off_a);   // planes k0.., row pitch rp, plane pitch pp
    T* B = reinterpret_cast<T*>(smem + E.off_b);
    T* G = reinterpret_cast<T*>(smem + E.off_g);   // this CTA's modes, index q N + k - 1
    T* Pv = reinterpret_cast<T*>(smem + E.off_p);
    const int k0 = cl_kfirst(r, C, nz), k1 = cl_kfirst(r + 1, C, nz);
    const int klo = max(1, k0), khi = min(nz - 1, k1 - 1);
    const int nk = max(0, khi - klo + 1);
    const int base = (klo - k0) * pp;   // first interior plane in A and B
    const int m0 = r * E.mm, nm = max(0, min(P, m0 + E.mm) - m0);
    const int nx4 = nx / 4;
    for (int q = t; q < 2 * nx * nx + 2 * ny * ny; q += bd) Qx[q] = E.Q[q];
    for (int q = t; q < nk * P; q += bd) {
        const int row = fdiv(q, E.f_x);   // kk ny + j
        A[base + row * rp + (q - row * nx)] = E.gf[(size_t)klo * P + q];
    }
    for (int q = t; q < nm * N; q += bd) Pv[q] = E.p[(size_t)m0 * N + q];
    __syncthreads();
    const int rows4 = nk * ny / 4;   // 4-row groups over all planes (ny is a multiple of 4)
    // forward along x: B[row][mx] = sum_i A[row][i] Qx[mx][i]
    for (int q = t; q < rows4 * nx4; q += bd) {
        const int rg = fdiv(q, E.f_x4), cg4 = q - rg * nx4;
        T acc[4][4];
        tile4<T, false>(A + base + 4 * rg * rp, 1, rp, QxT + 4 * cg4, nx, nx, acc);
#pragma unroll
        for (int a = 0; a < 4; ++a) st4(B + base + (4 * rg + a) * rp + 4 * cg4, acc[a]);
    }
    __syncthreads();
    // forward along y, times h^2: A[my][mx] = h^2 sum_j Qy[my][j] B[j][mx]
    for (int q = t; q < nk * (ny / 4) * nx4; q += bd) {
        const int kk = fdiv(q, E.f_t2), rem = q - kk * (ny / 4) * nx4;
        const int mg = fdiv(rem, E.f_x4), cg4 = rem - mg * nx4;
        T acc[4][4];
        tile4<T, true>(QyT + 4 * mg, ny, 0, B + base + kk * pp + 4 * cg4, rp, ny, acc);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] *= E.h2;
            st4(A + base + kk * pp + (4 * mg + a) * rp + 4 * cg4, acc[a]);
        }
    }
    cl.sync();
    // this CTA's modes: spectral right-hand sides from every plane's holder
    for (int q = t; q < nm * N; q += bd) {
        const int mq = fdiv(q, E.f_n);
        const int k = 1 + q - mq * N;
        const int o = cl_owner(k, C, nz);
        const int m = m0 + mq, my = fdiv(m, E.f_x);
        T* src = A + (k - cl_kfirst(o, C, nz)) * pp + my * rp + (m - my * nx);
        G[q] = *cl.map_shared_rank(src, o);
    }
    __syncthreads();
    for (int mq = t; mq < nm; mq += bd) {
        T* g = G + mq * N;
        const T* pv = Pv + mq * N;
        T acc = (T)0;
        for (int k = 0; k < N; ++k) {
            acc = (g[k] + acc) * pv[k];
            g[k] = acc;
        }
        T x = (T)0;
        for (int k = N - 1; k >= 0; --k) {
            x = g[k] + pv[k] * x;
            g[k] = x;
        }
    }
    __syncthreads();
    for (int q = t; q < nm * N; q += bd) {
        const int mq = fdiv(q, E.f_n);
        const int k = 1 + q - mq * N;
        const int o = cl_owner(k, C, nz);
        const int m = m0 + mq, my = fdiv(m, E.f_x);
        T* dst = A + (k - cl_kfirst(o, C, nz)) * pp + my * rp + (m - my * nx);
        *cl.map_shared_rank(dst, o) = G[q];
    }
    cl.sync();
    // inverse along y: B[j][mx] = sum_my Qy[my][j] A[my][mx]
    for (int q = t; q < nk * (ny / 4) * nx4; q += bd) {
        const int kk = fdiv(q, E.f_t2), rem = q - kk * (ny / 4) * nx4;
        const int jg = fdiv(rem, E.f_x4), cg4 = rem - jg * nx4;
        T acc[4][4];
        tile4<T, true>(Qy + 4 * jg, ny, 0, A + base + kk * pp + 4 * cg4, rp, ny, acc);
#pragma unroll
        for (int a = 0; a < 4; ++a) st4(B + base + kk * pp + (4 * jg + a) * rp + 4 * cg4, acc[a]);
    }
    __syncthreads();
    // inverse along x: u[row][i] = sum_mx B[row][mx] Qx[mx][i]
    for (int q = t; q < rows4 * nx4; q += bd) {
        const int rg = fdiv(q, E.f_x4), cg4 = q - rg * nx4;
        T acc[4][4];
        tile4<T, false>(B + base + 4 * rg * rp, 1, rp, Qx + 4 * cg4, nx, nx, acc);
#pragma unroll
        for (int a = 0; a < 4; ++a) st4(E.gu + (size_t)klo * P + (size_t)(4 * rg + a) * nx + 4 * cg4, acc[a]);
    }
}

// shared-memory layout of the exact solve of level l on C CTAs; false if it does not fit
template <typename T>
bool exact_layout(const pic_ctx* c, int l, int C, ExactLevel<T>* out, size_t* smem)
{
    const MGLevel& M = c->mg[l];
    ExactLevel<T> E{};
    E.nx = M.nx;
    E.ny = M.ny;
    E.nz = M.nz;
    E.rp = M.nx + 4;
    E.h2 = (T)(M.h * M.h);
    const int P = M.nx * M.ny, N = M.nz - 1;
    if (N < 1 || M.nz < C || M.nx % 4 != 0 || M.ny % 4 != 0) return false;
    E.mp = (M.nz + C - 1) / C + 1;
    E.mm = (P + C - 1) / C;
    auto al = [](size_t b) { return (b + 15) / 16 * 16; };
    const size_t plane = (size_t)M.ny * E.rp;
    size_t off = al(sizeof(T) * (2 * (size_t)M.nx * M.nx + 2 * (size_t)M.ny * M.ny));
    E.off_a = (unsigned int)off;
    off += al(sizeof(T) * (size_t)E.mp * plane);
    E.off_b = (unsigned int)off;
    off += al(sizeof(T) * (size_t)E.mp * plane);
    E.off_g = (unsigned int)off;
    off += al(sizeof(T) * (size_t)E.mm * N);
    E.off_p = (unsigned int)off;
    off += al(sizeof(T) * (size_t)E.mm * N);
    if (off > kClSmemMax) return false;
    E.Q = (const T*)c->ex_q;
    E.p = (const T*)c->ex_p;
    E.gf = (const T*)M.f;
    E.gu = (T*)M.u;
    E.f_x = fast_div(M.nx);
    E.f_n = fast_div(N);
    E.f_x4 = fast_div(M.nx / 4);
    E.f_y4 = fast_div(M.ny / 4);
    E.f_t2 = fast_div((M.ny / 4) * (M.nx / 4));
    if (out) *out = E;
    if (smem) *smem = off;
    return true;
}

template <typename T>
cudaError_t launch_exact(cudaStream_t s, const ExactLevel<T>& E, int C, size_t smem, bool query, int* fits)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)C, 1, 1);
    cfg.blockDim = dim3(kClThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (query) {
        cudaError_t e = cudaFuncSetAttribute(k_coarse_exact<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kClSmemMax);
        if (e == cudaSuccess && C > 8)
            e = cudaFuncSetAttribute(k_coarse_exact<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        int n = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, k_coarse_exact<T>, &cfg);
        *fits = e == cudaSuccess && n > 0;
        cudaGetLastError();
        return cudaSuccess;
    }
    return cudaLaunchKernelEx(&cfg, k_coarse_exact<T>, E);
}


// grid for kernels that reduce a norm: (x, y) blocks of a plane and just enough
// z blocks (each looping over planes) to fill the GPU a few times
inline Grid3 grid_norm(int nx, int ny, int planes)
{
    Grid3 g = grid3(nx, ny, 1);
    const int per_plane = (int)(g.grid.x * g.grid.y);
    // whole planes per block row, never more blocks than one resident wave: a
    // partial second wave of plane-looping blocks would double the kernel's time
    const int zb = std::max(1, std::min(planes, PIC_NORM_BLOCKS / per_plane));
    g.grid.z = (unsigned)zb;
    return g;
}

template <typename T>
void run_rbgs(cudaStream_t s, T* u, const T* f, Dims d, T h2, int color, int zero)
{
    if (d.half) {
        if (d.nx % 4 == 0 && d.half % 2 == 0) {
            Grid3 g = grid3(d.nx / 4, d.ny, 1);
            const int zp = column_planes(g, d.nz - 1, kRbPlanes);
            g.grid.z = (unsigned)std::max(1, (d.nz - 1 + zp - 1) / zp);
            launch_pdl(s, g.grid, g.block, k_rbgs_split2<T>, u, f, d, h2, color, zero, zp);
            return;
        }
        Grid3 g = grid3(d.nx / 2, d.ny, 1);
        const int zp = column_planes(g, d.nz - 1, kRbPlanes);
        g.grid.z = (unsigned)std::max(1, (d.nz - 1 + zp - 1) / zp);
        launch_pdl(s, g.grid, g.block, k_rbgs_split<T>, u, f, d, h2, color, zero, zp);
        return;
    }
    const Grid3 g = grid3(d.nx / 2, d.ny, d.nz - 1);
    launch_pdl(s, g.grid, g.block, k_rbgs<T>, u, f, d, h2, color, zero);
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
void run_resid_restrict(cudaStream_t s, const T* u, const T* f, T* fc, T* uc, Dims df, Dims dc, T inv_h2, T h2c,
                        T* rr = nullptr)
{
    if (df.half && rr && df.nx == 2 * dc.nx && df.ny == 2 * dc.ny && df.nz == 2 * dc.nz) {
        // split level: the red residuals in one pass, then the restriction
        if (df.nx % 4 == 0 && df.half % 2 == 0) {
            Grid3 g1 = grid3(df.nx / 4, df.ny, 1);
            const int zp = column_planes(g1, df.nz - 1, kRbPlanes);
            g1.grid.z = (unsigned)std::max(1, (df.nz - 1 + zp - 1) / zp);
            launch_pdl(s, g1.grid, g1.block, k_resid_red_split2<T>, u, f, rr, df, inv_h2, zp);
        } else {
            Grid3 g1 = grid3(df.nx / 2, df.ny, 1);
            const int zp = column_planes(g1, df.nz - 1, kRbPlanes);
            g1.grid.z = (unsigned)std::max(1, (df.nz - 1 + zp - 1) / zp);
            launch_pdl(s, g1.grid, g1.block, k_resid_red_split<T>, u, f, rr, df, inv_h2, zp);
        }
        const Grid3 g2 = grid3(dc.nx, dc.ny, dc.nz - 1);
        launch_pdl(s, g2.grid, g2.block, k_restrict_red<T>, (const T*)rr, fc, uc, df, dc, h2c);
        return;
    }
    const Grid3 g = grid3(dc.nx, dc.ny, dc.nz - 1);
    launch_pdl(s, g.grid, g.block, k_resid_restrict<T>, u, f, fc, uc, df, dc, inv_h2, h2c);
}
template <typename T>
void run_prolong(cudaStream_t s, T* uf, const T* uc, Dims df, Dims dc)
{
    if (df.nx == 2 * dc.nx && df.ny == 2 * dc.ny && df.nz == 2 * dc.nz) {
        if (df.half) {
            Grid3 g = grid3(dc.nx, dc.ny, 1);
            const int zp = column_planes(g, dc.nz, kSplitPlanes);
            g.grid.z = (unsigned)std::max(1, (dc.nz + zp - 1) / zp);
            launch_pdl(s, g.grid, g.block, k_prolong_split<T>, uf, uc, df, dc, zp);
            return;
        }
        const Grid3 g = grid3(dc.nx, dc.ny, dc.nz);
        launch_pdl(s, g.grid, g.block, k_prolong_cell<T>, uf, uc, df, dc);
        return;
    }
    const Grid3 g = grid3(df.nx, df.ny, df.nz - 1);
    launch_pdl(s, g.grid, g.block, k_prolong<T>, uf, uc, df, dc);
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

// One V-cycle from level l down on A e = f (f in mg[l].f); returns the array
// that holds the level's correction afterwards.
template <typename T>
T* vcycle(pic_ctx* c, int l)
{
    if (l == c->ex_level) {
        // this level is solved exactly
        ExactLevel<T> E{};
        size_t smem = 0;
        exact_layout<T>(c, l, c->ex_size, &E, &smem);
        int fits = 0;
        launch_exact<T>(c->stream, E, c->ex_size, smem, false, &fits);
        c->launches += 1;
        return (T*)c->mg[l].u;
    }
    if (l >= c->mg_tail) {
        // every level from here down runs in one cluster
        ClusterLevels<T> L{};
        size_t smem = 0;
        cluster_levels<T>(c, l, c->cl_size, &L, &smem);
        int fits = 0;
        launch_cluster<T>(c->stream, L, c->cl_size, smem, false, &fits);
        c->launches += 1;
        return (T*)c->mg[l].u;
    }
    MGLevel& L = c->mg[l];
    const Dims d{L.nx, L.ny, L.nz, L.half};
    const T h2 = (T)(L.h * L.h);
    T* u = (T*)L.u;
    T* f = (T*)L.f;
    // pre-smoothing from a zero guess: the first red pass needs no neighbours
    // (on the coarser levels the restriction above has already made it)
    for (int s = 0; s < kPre; ++s)
        for (int color = 0; color < 2; ++color) {
            if (s == 0 && color == 0 && l > 0) continue;
            run_rbgs<T>(c->stream, u, f, d, h2, color, s == 0 && color == 0);
            c->launches += 1;
        }
    MGLevel& C = c->mg[l + 1];
    const Dims dc{C.nx, C.ny, C.nz, C.half};
    run_resid_restrict<T>(c->stream, u, f, (T*)C.f, (T*)C.u, d, dc, (T)(1.0 / (L.h * L.h)), (T)(C.h * C.h),
                          (T*)L.r);
    c->launches += d.half ? 2 : 1;
    T* uc = vcycle<T>(c, l + 1);
    run_prolong<T>(c->stream, u, (const T*)uc, d, dc);
    c->launches += 1 + 2 * kPost;
    for (int s = 0; s < kPost; ++s)
        for (int color = 0; color < 2; ++color) run_rbgs<T>(c->stream, u, f, d, h2, color, 0);
    return u;
}

template <typename T>
pic_status solve_t(pic_ctx* c, double tol, int max_iters, int* iters, double* res)
{
    const Dims d{c->nx, c->ny, c->nz, c->mg[0].half};   // mg[0].f receives the residual
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
        const T* e = vcycle<T>(c, 0);
        cudaMemsetAsync(c->d_norm + 1, 0, sizeof(double), c->stream);
        run_resid64<T>(c->stream, c->phi, e, c->f64, c->phi_alt, (T*)L0.f, c->d_norm + 1, d, inv_h2);
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
    const Dims d{c->nx, c->ny, c->nz, c->mg[0].half};   // mg[0].f receives the residual
    const T* e = vcycle<T>(c, 0);
    const Grid3 g = grid3(d.nx, d.ny, d.nz - 1);
    k_add<T><<<g.grid, g.block, 0, c->stream>>>(c->phi, e, d);
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
    const Dims d{c->nx, c->ny, c->nz, c->mg[0].half};   // mg[0].f receives the residual
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

// ---- mixed precision: the refinement in double-float arithmetic -----------
// FP64 instructions issue at about 1/70 of the FP32 rate on this GPU, so the
// mixed solver keeps the potential and the right-hand side as unevaluated sums
// hi + lo of two floats (about 48 significant bits) and forms the residual
// with error-free transformations in FP32: Knuth's TwoSum, Dekker's Fast2Sum
// and the exact product a*b = p + fma(a, b, -p).  The potential lives in two
// buffers; an iteration reads one and writes phi + e into the other, so the
// correction and the residual of the updated potential take one pass.

// s + e == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// s + e == a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    e = b - (s - a);
}
__device__ __forceinline__ float2 df_add_f(float2 a, float b)
{
    float s, e, h, l;
    two_sum(a.x, b, s, e);
    e += a.y;
    fast_two_sum(s, e, h, l);
    return make_float2(h, l);
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b)
{
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e += a.x * b.y + a.y * b.x;
    float h, l;
    fast_two_sum(p, e, h, l);
    return make_float2(h, l);
}
__host__ __device__ inline float2 df_of(double v)
{
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}
// a 64-bit integer as hi + lo: three exact pieces of at most 24 bits
__device__ __forceinline__ float2 df_of_i64(long long v)
{
    const float a = (float)(int)(v >> 40) * 0x1p40f;
    const float b = (float)(int)((v >> 20) & 0xFFFFF) * 0x1p20f;
    const float c = (float)(int)(v & 0xFFFFF);
    float s, e, s2, e2, h, l;
    two_sum(a, b, s, e);
    two_sum(s, c, s2, e2);
    fast_two_sum(s2, e2 + e, h, l);
    return make_float2(h, l);
}

__device__ __forceinline__ float block_sum_f(float v)
{
    __shared__ float part[32];
    const int t = tid_flat(), nt = blockDim.x * blockDim.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = t & 31, w = t >> 5;
    if (lane == 0) part[w] = v;
    __syncthreads();
    v = (t < (nt + 31) / 32) ? part[t] : 0.f;
    if (w == 0)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Grid-wide sum of one value per thread without atomics on the sum: each
// block stores its partial, the last block to arrive (one counter increment
// per block) adds the partials in block order.  Returns true in the last
// block, whose threads all receive the total.  The counter wraps back to 0.
__device__ bool grid_sum_last(float v, float* part, unsigned int* count, float& total)
{
    __shared__ int s_last;
    __shared__ float s_tot;
    v = block_sum_f(v);
    const int t = tid_flat();
    const unsigned int nb = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (t == 0) {
        part[b] = v;
        __threadfence();
        s_last = atomicInc(count, nb - 1) == nb - 1;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    float acc = 0.f;
    for (unsigned int q = t; q < nb; q += blockDim.x * blockDim.y) acc += __ldcg(part + q);
    acc = block_sum_f(acc);
    if (t == 0) s_tot = acc;
    __syncthreads();
    total = s_tot;
    return true;
}

struct RhsDf {
    float2* phi;                     // two buffers of nodes; buffer 0 holds the warm start
    float2* F;                       // out: h^2 rho / eps0
    const unsigned long long* rq;
    float* part;
    DfState* st;
    double* vb_last;                 // lower electrode value of the previous solve (null: no shift)
    const uint32_t* step;            // device step counter: electrode values from the drive, else vb, vt
    SolveParams sp;
    double scale, vb, vt, h2;
};

// Head of a mixed-precision solve, one thread per node of planes 0..nz:
// F = h^2 rho / eps0 from the fixed-point charge, electrode values on both
// buffers, the warm start moved by the change of the electrode ramp
// (vb - vb_last)(1 - z / Lz), which the 7-point operator maps to zero, and
// ||h^2 b||^2 (b = f plus the electrode terms next to the planes).
__global__ void __launch_bounds__(256) k_rhs_df(RhsDf a, Dims d)
{
    __shared__ float2 s_vb, s_vt, s_sc;
    __shared__ float s_shift;
    __shared__ double s_vbd;
    if (tid_flat() == 0) {
        double vb = a.vb, vt = a.vt, sc = a.scale;
        if (a.step) {
            vb = bottom_potential(a.sp, *a.step);
            vt = a.sp.v_top;
            sc = a.sp.scale;
        }
        s_vbd = vb;
        s_vb = df_of(vb);
        s_vt = df_of(vt);
        s_sc = df_of(sc * a.h2);
        s_shift = a.vb_last ? (float)(vb - *a.vb_last) : 0.f;
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const size_t N = (size_t)d.nx * d.ny * (d.nz + 1);
    float acc = 0.f;
    if (i < d.nx && j < d.ny)
        for (int k = blockIdx.z; k <= d.nz; k += gridDim.z) {
            const int n = (k * d.ny + j) * d.nx + i;
            const float2 F = df_mul(df_of_i64((long long)a.rq[n]), s_sc);
            a.F[n] = F;
            if (k == 0) {
                a.phi[n] = s_vb;
                a.phi[N + n] = s_vb;
            } else if (k == d.nz) {
                a.phi[n] = s_vt;
                a.phi[N + n] = s_vt;
            } else {
                if (s_shift != 0.f) a.phi[n] = df_add_f(a.phi[n], s_shift * (1.f - (float)k / (float)d.nz));
                float b = F.x + F.y;
                if (k == 1) b += s_vb.x;
                if (k == d.nz - 1) b += s_vt.x;
                acc += b * b;
            }
        }
    float b2;
    if (!grid_sum_last(acc, a.part, &a.st->cnt_head, b2)) return;
    if (tid_flat() == 0) {
        a.st->b2 = b2;
        a.st->sel = 0;
        if (a.vb_last) *a.vb_last = s_vbd;
    }
}

struct ResDf {
    float2* phi;                     // two buffers of nodes
    const float* e;                  // V-cycle correction on the fine level (null: none, nothing written)
    const float2* F;
    float* r;                        // out: r = R / h^2, the next V-cycle's right-hand side
    float* part;
    DfState* st;
    unsigned int* iters;
    double* res;
    int* flag;                       // latch for a failed graph solve (null in host-driven solves)
    unsigned long long* total;
    float inv_h2, tol2, h4;
    int max_iters, first, use_cond;
    cudaGraphConditionalHandle h;
};

// One refinement step over the interior nodes: phi' = phi + e (written to the
// other buffer), R = h^2 f - (6 phi' - sum of the 6 neighbours of phi') with
// the large parts summed exactly, ||R||^2 over the grid, and in the last block
// the loop decision of the solve (the same rule as the FP64 solver's).
// the refinement step: most planes per block (a 32 x 8 column tile of them) and
// resident blocks per SM it is built for
constexpr int kResidPlanes = 16;
constexpr int kResidBlocks = 4;

// the potential (hi + lo) and the V-cycle correction at one node
struct PhiE {
    float2 p;
    float e;
};

// R = h^2 f - (6 phi'_n - sum of the 6 neighbours' phi') at one node, phi' =
// phi + e, and phi'_n itself (to `out`); neighbours in the order x+, x-, y+,
// y-, z+, z-.  kF64: the residual formed in FP64 arithmetic from the
// two-float values (the measured alternative to the double-float sums).
template <bool kF64>
__device__ __forceinline__ float node_resid(const PhiE& c, const PhiE (&nb)[6], float2 F, float2& out)
{
    if (kF64) {
        const double pd = ((double)c.p.x + (double)c.p.y) + (double)c.e;
        double lap = 6.0 * pd;
#pragma unroll
        for (int q = 0; q < 6; ++q) lap -= ((double)nb[q].p.x + (double)nb[q].p.y) + (double)nb[q].e;
        out = df_of(pd);
        return (float)(((double)F.x + (double)F.y) - lap);
    }
    // 6 phi'_n - sum phi'_nb: hi parts exactly (s + err), the small parts in float
    float sh = 6.f * c.p.x;
    float err = fmaf(6.f, c.p.x, -sh);
    float small = 6.f * (c.p.y + c.e);
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        float s2, t;
        two_sum(sh, -nb[q].p.x, s2, t);
        sh = s2;
        err += t;
        small -= nb[q].p.y + nb[q].e;
    }
    float r1, t1;
    two_sum(F.x, -sh, r1, t1);
    out = df_add_f(c.p, c.e);
    return r1 + ((t1 + F.y) - (err + small));
}

// the end of a refinement step: ||R||^2 over the grid and, in the last block,
// the loop decision of the solve (the same rule as the FP64 solver's)
__device__ __forceinline__ void resid_df_tail(const ResDf& a, float acc, int sel)
{
    float r2;
    if (!grid_sum_last(acc, a.part, &a.st->cnt_res, r2)) return;
    if (tid_flat() != 0) return;
    const float b2 = a.st->b2;
    const float target2 = a.tol2 * (b2 > 0.f ? b2 : a.h4);
    const unsigned int it = a.first ? 0u : *a.iters + 1u;
    *a.iters = it;
    if (!a.first) *a.total += 1ull;
    const bool ok = r2 <= target2;
    const bool finite = isfinite(r2);
    const bool more = !ok && finite && (int)it < a.max_iters;
    *a.res = b2 > 0.f ? sqrt((double)r2 / (double)b2) : sqrt((double)r2 / (double)a.h4);
    const int status = ok ? (int)PIC_OK : finite ? (int)PIC_ENOTCONV : (int)PIC_ENONFINITE;
    if (!more && !ok && a.flag) atomicCAS(a.flag, 0, status);
    a.st->status = status;
    a.st->more = more ? 1 : 0;
    if (a.e) a.st->sel = sel ^ 1;
    if (a.use_cond) cudaGraphSetConditional(a.h, more ? 1u : 0u);
}

// One refinement step over the interior nodes: phi' = phi + e (written to the
// other buffer), R = h^2 f - (6 phi' - sum of the 6 neighbours of phi') with
// the large parts summed exactly, ||R||^2 over the grid, and the loop decision.
// Natural layout of e and r; thread (i, j) walks zp planes of its
// column: the values at k - 1, k and k + 1 roll through registers, and the
// loads for plane k + 1 (its in-plane neighbours and f, the column at k + 2)
// are issued before plane k is computed.  The potential, correction and f are
// only read here (the new potential goes to the other buffer), so the loads
// take the read-only path.
template <bool kF64>
__global__ void __launch_bounds__(256, kResidBlocks) k_resid_df(ResDf a, Dims d, int zp)
{
    pdl_begin();
    __shared__ int s_sel;
    if (tid_flat() == 0) s_sel = a.st->sel;
    __syncthreads();
    const size_t N = (size_t)d.nx * d.ny * (d.nz + 1);
    const float2* cur = a.phi + (s_sel ? N : 0);
    float2* nxt = a.phi + (s_sel ? 0 : N);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = 1 + (int)blockIdx.z * zp;
    const int k1 = min(k0 + zp, d.nz);
    float acc = 0.f;
    if (i < d.nx && j < d.ny && k0 < k1) {
        const int P = d.nx * d.ny;
        const int off[4] = {(i + 1 == d.nx) ? 1 - d.nx : 1, (i == 0) ? d.nx - 1 : -1,
                            (j + 1 == d.ny) ? -j * d.nx : d.nx, (j == 0) ? (d.ny - 1) * d.nx : -d.nx};
        auto ld = [&](int n) {
            PhiE v;
            v.p = __ldg(cur + n);
            v.e = a.e ? __ldg(a.e + n) : 0.f;
            return v;
        };
        int n = (k0 * d.ny + j) * d.nx + i;
        PhiE zm = ld(n - P), zc = ld(n), zp = ld(n + P);
        PhiE X[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) X[q] = ld(n + off[q]);
        float2 F = __ldg(a.F + n);
        for (int k = k0; k < k1; ++k, n += P) {
            PhiE Xn[4], zn = zp;
            float2 Fn = F;
            if (k + 1 < k1) {
                zn = ld(n + 2 * P);
#pragma unroll
                for (int q = 0; q < 4; ++q) Xn[q] = ld(n + P + off[q]);
                Fn = __ldg(a.F + n + P);
            }
            const PhiE nbv[6] = {X[0], X[1], X[2], X[3], zp, zm};
            float2 upd;
            const float R = node_resid<kF64>(zc, nbv, F, upd);
            if (a.e) nxt[n] = upd;
            a.r[n] = R * a.inv_h2;
            acc += R * R;
            zm = zc;
            zc = zp;
            zp = zn;
#pragma unroll
            for (int q = 0; q < 4; ++q) X[q] = Xn[q];
            F = Fn;
        }
    }
    resid_df_tail(a, acc, s_sel);
}

// The same step on a red-black split finest level (d.half > 0: e and r split
// by colour, the potential and f in natural order), by columns of node pairs:
// thread (i2, j) takes nodes 2 i2 and 2 i2 + 1 of each row (j, k) of its
// zp planes, their potential and f as one 16-byte load each, their
// corrections at pair index m in the red and black halves.  Each node's
// neighbours are those of k_resid_df, in its order; the pairs at k - 1, k and
// k + 1 roll through registers, the one at k + 2 is loaded a plane ahead.
struct PairPE {
    float4 p;       // the two nodes' potentials (hi, lo, hi, lo)
    float e0, e1;   // their corrections
};

template <bool kF64>
__global__ void __launch_bounds__(256, kResidBlocks) k_resid_df_pairs(ResDf a, Dims d, int zp)
{
    pdl_begin();
    __shared__ int s_sel;
    if (tid_flat() == 0) s_sel = a.st->sel;
    __syncthreads();
    const size_t N = (size_t)d.nx * d.ny * (d.nz + 1);
    const float2* cur = a.phi + (s_sel ? N : 0);
    float2* nxt = a.phi + (s_sel ? 0 : N);
    const int hx = d.nx >> 1, P2 = hx * d.ny, P = d.nx * d.ny;
    const int i2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = 1 + (int)blockIdx.z * zp;
    const int k1 = min(k0 + zp, d.nz);
    float acc = 0.f;
    if (i2 < hx && j < d.ny && k0 < k1) {
        const float* eR = a.e;
        const float* eB = a.e ? a.e + d.half : nullptr;
        // the pair at natural node n (even) and pair index m; c0 = colour of its node 0
        auto ldp = [&](int n, int m, int c0) {
            PairPE v;
            v.p = __ldg(reinterpret_cast<const float4*>(cur + n));
            v.e0 = a.e ? __ldg((c0 ? eB : eR) + m) : 0.f;
            v.e1 = a.e ? __ldg((c0 ? eR : eB) + m) : 0.f;
            return v;
        };
        // one node (float2 at natural n, correction of colour col at pair m)
        auto ld1 = [&](int n, int m, int col) {
            PhiE v;
            v.p = __ldg(cur + n);
            v.e = a.e ? __ldg((col ? eB : eR) + m) : 0.f;
            return v;
        };
        const int dxp = (i2 + 1 == hx) ? 1 - hx : 1, dxm = (i2 == 0) ? hx - 1 : -1;
        const int dyp = (j + 1 == d.ny) ? -j * hx : hx, dym = (j == 0) ? (d.ny - 1) * hx : -hx;
        int m = k0 * P2 + j * hx + i2;
        int n = 2 * m;   // natural index of node 0 (nx even: n = k P + j nx + 2 i2)
        int c0 = (j + k0) & 1;
        PairPE zm = ldp(n - P, m - P2, c0 ^ 1), zc = ldp(n, m, c0), zp = ldp(n + P, m + P2, c0 ^ 1);
        for (int k = k0; k < k1; ++k, m += P2, n += P, c0 ^= 1) {
            PairPE zn = zp;
            if (k + 1 < k1) zn = ldp(n + 2 * P, m + 2 * P2, c0);
            const PairPE yp = ldp(n + 2 * dyp, m + dyp, c0 ^ 1), ym = ldp(n + 2 * dym, m + dym, c0 ^ 1);
            // x- of node 0: node 1 of the pair on the left (colour c0 ^ 1); x+ of
            // node 1: node 0 of the pair on the right (colour c0)
            const PhiE xl = ld1(n + 2 * dxm + 1, m + dxm, c0 ^ 1), xr = ld1(n + 2 * dxp, m + dxp, c0);
            const float4 F = __ldg(reinterpret_cast<const float4*>(a.F + n));
            const PhiE n0{make_float2(zc.p.x, zc.p.y), zc.e0}, n1{make_float2(zc.p.z, zc.p.w), zc.e1};
            const PhiE nb0[6] = {n1,
                                 xl,
                                 {make_float2(yp.p.x, yp.p.y), yp.e0},
                                 {make_float2(ym.p.x, ym.p.y), ym.e0},
                                 {make_float2(zp.p.x, zp.p.y), zp.e0},
                                 {make_float2(zm.p.x, zm.p.y), zm.e0}};
            const PhiE nb1[6] = {xr,
                                 n0,
                                 {make_float2(yp.p.z, yp.p.w), yp.e1},
                                 {make_float2(ym.p.z, ym.p.w), ym.e1},
                                 {make_float2(zp.p.z, zp.p.w), zp.e1},
                                 {make_float2(zm.p.z, zm.p.w), zm.e1}};
            float2 u0, u1;
            const float R0 = node_resid<kF64>(n0, nb0, make_float2(F.x, F.y), u0);
            const float R1 = node_resid<kF64>(n1, nb1, make_float2(F.z, F.w), u1);
            if (a.e) *reinterpret_cast<float4*>(nxt + n) = make_float4(u0.x, u0.y, u1.x, u1.y);
            (c0 ? a.r + d.half : a.r)[m] = R0 * a.inv_h2;
            (c0 ? a.r : a.r + d.half)[m] = R1 * a.inv_h2;
            acc += R0 * R0;
            acc += R1 * R1;
            zm = zc;
            zc = zp;
            zp = zn;
        }
    }
    resid_df_tail(a, acc, s_sel);
}

// after the loop: the current potential back into buffer 0
__global__ void k_settle_df(float2* phi, const DfState* st, size_t N)
{
    pdl_begin();
    if (st->sel == 0) return;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x)
        phi[n] = phi[N + n];
}

__global__ void k_df_to_f64(const float2* __restrict__ phi2, double* __restrict__ phi, size_t N)
{
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const float2 p = phi2[n];
        phi[n] = (double)p.x + (double)p.y;
    }
}

__global__ void k_f64_to_df(const double* __restrict__ phi, float2* __restrict__ phi2, size_t N)
{
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x)
        phi2[n] = df_of(phi[n]);
}

// head kernel; step != null takes the electrode values and scale from the device step
void launch_rhs_df(pic_ctx* c, const uint32_t* step, double scale, double vb, double vt, bool warm_shift)
{
    const Dims d{c->nx, c->ny, c->nz};
    RhsDf a{};
    a.phi = c->phi2;
    a.F = c->f2;
    a.rq = c->rq;
    a.part = c->d_part;
    a.st = c->d_dfs;
    a.vb_last = warm_shift ? c->d_vb_last : nullptr;
    a.step = step;
    a.sp = c->sp;
    a.scale = scale;
    a.vb = vb;
    a.vt = vt;
    a.h2 = c->dx * c->dx;
    const Grid3 g = grid_norm(d.nx, d.ny, d.nz + 1);
    k_rhs_df<<<g.grid, g.block, 0, c->stream>>>(a, d);
    c->launches += 1;
}

void launch_resid_df(pic_ctx* c, double tol, int max_iters, const float* e, bool graph, cudaGraphConditionalHandle h)
{
    const Dims d{c->nx, c->ny, c->nz, c->mg[0].half};   // mg[0].f receives the residual
    ResDf a{};
    a.phi = c->phi2;
    const bool first = e == nullptr;
    a.e = e;
    a.F = c->f2;
    a.r = (float*)c->mg[0].f;
    a.part = c->d_part;
    a.st = c->d_dfs;
    a.iters = c->d_iters;
    a.res = c->d_res;
    a.flag = graph ? c->d_solve_flag : nullptr;
    a.total = c->d_iter_total;
    a.inv_h2 = (float)(1.0 / (c->dx * c->dx));
    a.tol2 = (float)(tol * tol);
    a.h4 = (float)(c->dx * c->dx * c->dx * c->dx);
    a.max_iters = max_iters;
    a.first = first ? 1 : 0;
    a.use_cond = graph ? 1 : 0;
    a.h = h;
    const bool f64 = (c->flags & PIC_F_F64_RESIDUAL) != 0;
    Grid3 g = grid3(d.half ? d.nx / 2 : d.nx, d.ny, 1);
    const int zp = column_planes(g, d.nz - 1, kResidPlanes);
    g.grid.z = (unsigned)std::max(1, (d.nz - 1 + zp - 1) / zp);
    if (d.half) {
        if (f64) launch_pdl(c->stream, g.grid, g.block, k_resid_df_pairs<true>, a, d, zp);
        else launch_pdl(c->stream, g.grid, g.block, k_resid_df_pairs<false>, a, d, zp);
    } else {
        if (f64) launch_pdl(c->stream, g.grid, g.block, k_resid_df<true>, a, d, zp);
        else launch_pdl(c->stream, g.grid, g.block, k_resid_df<false>, a, d, zp);
    }
    c->launches += 1;
}

void launch_settle_df(pic_ctx* c)
{
    k_settle_df<<<grid_for((int64_t)c->nodes, 256, 152 * 4), 256, 0, c->stream>>>(c->phi2, c->d_dfs, c->nodes);
    c->launches += 1;
}

// host-driven mixed solve after launch_rhs_df: loop decisions read back each iteration
pic_status solve_df(pic_ctx* c, double tol, int max_iters, int* iters, double* res)
{
    cudaGraphConditionalHandle none{};
    launch_resid_df(c, tol, max_iters, nullptr, false, none);
    DfState st{};
    while (true) {
        if (!PIC_CUDA_OK(cudaMemcpyAsync(&st, c->d_dfs, sizeof st, cudaMemcpyDeviceToHost, c->stream)) ||
            !PIC_CUDA_OK(cudaStreamSynchronize(c->stream)))
            return PIC_ECUDA;
        if (!st.more) break;
        const float* e = vcycle<float>(c, 0);
        launch_resid_df(c, tol, max_iters, e, false, none);
    }
    launch_settle_df(c);
    unsigned int it = 0;
    double rel = 0.0;
    if (!PIC_CUDA_OK(cudaMemcpyAsync(&it, c->d_iters, sizeof it, cudaMemcpyDeviceToHost, c->stream)) ||
        !PIC_CUDA_OK(cudaMemcpyAsync(&rel, c->d_res, sizeof rel, cudaMemcpyDeviceToHost, c->stream)) ||
        !PIC_CUDA_OK(cudaStreamSynchronize(c->stream)))
        return PIC_ECUDA;
    if (iters) *iters = (int)it;
    if (res) *res = rel;
    c->last_iters = it;
    c->last_res = rel;
    return (pic_status)st.status;
}

}  // namespace

void enqueue_solve_head(pic_ctx* c, double tol, int max_iters, cudaGraphConditionalHandle h)
{
    if (c->prec == PIC_MIXED) {
        launch_rhs_df(c, c->d_step, 0.0, 0.0, 0.0, true);
        launch_resid_df(c, tol, max_iters, nullptr, true, h);
    } else {
        enqueue_head<double>(c, tol, max_iters, h);
    }
}

void enqueue_solve_iteration(pic_ctx* c, double tol, int max_iters, cudaGraphConditionalHandle h)
{
    if (c->prec == PIC_MIXED) {
        const float* e = vcycle<float>(c, 0);
        launch_resid_df(c, tol, max_iters, e, true, h);
    } else {
        enqueue_iteration<double>(c, tol, max_iters, h);
    }
}

void enqueue_solve_tail(pic_ctx* c)
{
    if (c->prec == PIC_MIXED) launch_settle_df(c);
}

void phi_sync_f64(pic_ctx* c)
{
    if (c->prec != PIC_MIXED) return;
    k_df_to_f64<<<grid_for((int64_t)c->nodes, 256, 152 * 4), 256, 0, c->stream>>>(c->phi2, c->phi, c->nodes);
    c->launches += 1;
}

void phi_from_f64(pic_ctx* c)
{
    if (c->prec != PIC_MIXED) return;
    k_f64_to_df<<<grid_for((int64_t)c->nodes, 256, 152 * 4), 256, 0, c->stream>>>(c->phi, c->phi2, c->nodes);
    c->launches += 1;
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
    // the levels from mg_tail down run in one thread-block cluster from shared
    // memory: the first level (smallest index) that fits, with the largest
    // cluster the device can hold; larger levels run as grid-wide launches
    {
        int sizes[6] = {PIC_MG_CLUSTER, 16, 8, 4, 2, 1};
        bool found = false;
        for (int l0 = std::min(std::max(0, PIC_MG_CLUSTER_FROM), (int)c->mg.size() - 1); l0 < (int)c->mg.size() && !found;
             ++l0)
            for (int C : sizes) {
                if (C < 1 || C > 16 || C > PIC_MG_CLUSTER) continue;
                size_t smem = 0;
                const bool ok = c->prec == PIC_MIXED ? cluster_levels<float>(c, l0, C, nullptr, &smem)
                                                     : cluster_levels<double>(c, l0, C, nullptr, &smem);
                if (!ok) continue;
                int fits = 0;
                if (c->prec == PIC_MIXED) launch_cluster<float>(nullptr, ClusterLevels<float>{}, C, smem, true, &fits);
                else launch_cluster<double>(nullptr, ClusterLevels<double>{}, C, smem, true, &fits);
                if (!fits) continue;
                c->mg_tail = l0;
                c->cl_size = C;
                found = true;
                break;
            }
        if (!found) return PIC_ECUDA;
    }
    // the finest level below the first that one cluster can solve exactly
    c->ex_level = -1;
    for (int l = 1; PIC_MG_EXACT && l < (int)c->mg.size() && c->ex_level < 0; ++l)
        for (int C : {16, 8, 4, 2, 1}) {
            if (C > PIC_MG_CLUSTER) continue;
            if (c->mg[l].nodes > (size_t)PIC_MG_EXACT_MAXNODES) break;
            size_t smem = 0;
            const bool ok = c->prec == PIC_MIXED ? exact_layout<float>(c, l, C, nullptr, &smem)
                                                 : exact_layout<double>(c, l, C, nullptr, &smem);
            if (!ok) continue;
            int fits = 0;
            if (c->prec == PIC_MIXED) launch_exact<float>(nullptr, ExactLevel<float>{}, C, smem, true, &fits);
            else launch_exact<double>(nullptr, ExactLevel<double>{}, C, smem, true, &fits);
            if (!fits) continue;
            c->ex_level = l;
            c->ex_size = C;
            break;
        }
    // Red-black split layout (every kernel indexes such a level through lix):
    // the finest level when it runs as grid-wide launches, and each coarser
    // grid-wide level reached from a split level by halving every axis (the
    // restriction onto it and the prolongation from it then take the split
    // kernels, which read and write it by colour).
    for (int l = 0; l < (int)c->mg.size(); ++l) {
        MGLevel& M = c->mg[l];
        bool split = l < c->mg_tail && (c->ex_level < 0 || l < c->ex_level) && l + 1 < (int)c->mg.size() &&
                     M.nx % 2 == 0;
        if (l > 0) {
            const MGLevel& F = c->mg[l - 1];
            split = split && F.half > 0 && F.nx == 2 * M.nx && F.ny == 2 * M.ny && F.nz == 2 * M.nz;
        }
        M.half = split ? (int)(M.nodes / 2) : 0;
    }
    if (c->ex_level >= 0) {
        const MGLevel& M = c->mg[c->ex_level];
        // orthonormal real Fourier basis of length n (rows) and the eigenvalue of
        // the periodic second difference on each row
        auto basis = [](int n, std::vector<double>& q, std::vector<double>& lam) {
            q.assign((size_t)n * n, 0.0);
            lam.assign(n, 0.0);
            for (int i = 0; i < n; ++i) q[i] = 1.0 / std::sqrt((double)n);
            for (int p = 1; 2 * p < n; ++p) {
                const double a = 2.0 * kPI * p / n, w = std::sqrt(2.0 / n);
                for (int i = 0; i < n; ++i) {
                    q[(size_t)(2 * p - 1) * n + i] = w * std::cos(a * i);
                    q[(size_t)(2 * p) * n + i] = w * std::sin(a * i);
                }
                lam[2 * p - 1] = lam[2 * p] = 2.0 - 2.0 * std::cos(a);
            }
            if (n % 2 == 0) {
                for (int i = 0; i < n; ++i) q[(size_t)(n - 1) * n + i] = (i % 2 ? -1.0 : 1.0) / std::sqrt((double)n);
                lam[n - 1] = 4.0;
            }
        };
        std::vector<double> qx, lx, qy, ly;
        basis(M.nx, qx, lx);
        basis(M.ny, qy, ly);
        std::vector<double> qall;
        qall.insert(qall.end(), qx.begin(), qx.end());
        for (int i = 0; i < M.nx; ++i)
            for (int m = 0; m < M.nx; ++m) qall.push_back(qx[(size_t)m * M.nx + i]);
        qall.insert(qall.end(), qy.begin(), qy.end());
        for (int j = 0; j < M.ny; ++j)
            for (int m = 0; m < M.ny; ++m) qall.push_back(qy[(size_t)m * M.ny + j]);
        const int N = M.nz - 1;
        std::vector<double> piv((size_t)M.nx * M.ny * N);
        for (int my = 0; my < M.ny; ++my)
            for (int mx = 0; mx < M.nx; ++mx) {
                const double d = 2.0 + lx[mx] + ly[my];
                double pk = 0.0;
                for (int k = 0; k < N; ++k) {
                    pk = 1.0 / (d - pk);
                    piv[((size_t)my * M.nx + mx) * N + k] = pk;
                }
            }
        c->ex_q = dev_alloc(c, tsz * qall.size());
        c->ex_p = dev_alloc(c, tsz * piv.size());
        if (!c->ex_q || !c->ex_p) return PIC_ENOMEM;
        cudaError_t e;
        if (c->prec == PIC_MIXED) {
            std::vector<float> a(qall.begin(), qall.end()), b(piv.begin(), piv.end());
            e = cudaMemcpy(c->ex_q, a.data(), sizeof(float) * a.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(c->ex_p, b.data(), sizeof(float) * b.size(), cudaMemcpyHostToDevice);
        } else {
            e = cudaMemcpy(c->ex_q, qall.data(), sizeof(double) * qall.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(c->ex_p, piv.data(), sizeof(double) * piv.size(), cudaMemcpyHostToDevice);
        }
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
    if (c->prec == PIC_MIXED) {
        // double-float potential (two buffers), right-hand side, block partials, state
        const Grid3 g = grid3(c->nx, c->ny, c->nz + 1);
        const size_t parts = (size_t)g.grid.x * g.grid.y * g.grid.z;
        c->phi2 = (float2*)dev_alloc(c, sizeof(float2) * 2 * c->nodes);
        c->f2 = (float2*)dev_alloc(c, sizeof(float2) * c->nodes);
        c->d_part = (float*)dev_alloc(c, sizeof(float) * parts);
        c->d_dfs = (DfState*)dev_alloc(c, sizeof(DfState));
        if (!c->phi2 || !c->f2 || !c->d_part || !c->d_dfs) return PIC_ENOMEM;
        if (cudaMemset(c->phi2, 0, sizeof(float2) * 2 * c->nodes) != cudaSuccess ||
            cudaMemset(c->f2, 0, sizeof(float2) * c->nodes) != cudaSuccess ||
            cudaMemset(c->d_dfs, 0, sizeof(DfState)) != cudaSuccess)
            return PIC_ECUDA;
    }
    return PIC_OK;
}

void launch_rhs(pic_ctx* c, double scale, double v_bot, double v_top, bool warm_shift)
{
    if (c->prec == PIC_MIXED) {
        launch_rhs_df(c, nullptr, scale, v_bot, v_top, warm_shift);
        return;
    }
    const Dims d{c->nx, c->ny, c->nz};
    cudaMemsetAsync(c->d_norm, 0, sizeof(double), c->stream);
    const Grid3 g = grid_norm(d.nx, d.ny, d.nz + 1);
    k_rhs<<<g.grid, g.block, 0, c->stream>>>(c->rq, scale, c->f64, c->phi, c->phi_alt, v_bot, v_top, d,
                                            1.0 / (c->dx * c->dx), c->d_norm, warm_shift ? c->d_vb_last : nullptr);
    c->launches += 1;
    if (warm_shift) {
        k_store<<<1, 1, 0, c->stream>>>(c->d_vb_last, v_bot);
        c->launches += 1;
    }
}

pic_status mg_solve(pic_ctx* c, double, double, double tol, int max_iters, int* iters, double* res)
{
    if (c->prec == PIC_MIXED) return solve_df(c, tol, max_iters, iters, res);
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
constexpr size_t kNaMaxCoarse = 4096;        // largest coarsest level (red-black sweeps in one block)
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
    if (c.lv[c.nl - 1].nodes > kNaMaxCoarse) {
        // halving stops at the first level with nx or ny not divisible by 4, or nz odd or below 4; the
        // one-block smoother of the coarsest level is only exact enough on a small level
        set_global_error("pic_solve_noalloc: the mesh coarsens only to a level of more than 4096 nodes; halving "
                         "needs nx, ny divisible by 4 and nz even and >= 4 at each level");
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

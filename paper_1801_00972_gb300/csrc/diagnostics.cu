// Diagnostics beyond the step.
//
// Electron energy probability function (Sec. IV.A, Fig. 3): an exact integer
// histogram of electron energies per cell plane, accumulated every step after
// the collisions, and the two-Maxwellian fit the paper applies to it.
//
// A step adds one count per live electron to (its cell plane k, energy bin
// floor(eps / de)), eps = (m_e/2)|v|^2/e in eV; energies past the last bin go
// to an overflow bin.  The FP64 kernel takes the bin decision in FP64 exactly
// as the oracle does (this unit is built without fused multiply-add); the mixed
// kernel takes it in float from the cells/step velocities.
//
// Phase-resolved moments and the fine MD-region grid (Sec. IV.C): each moment
// sample goes into the rf phase bin of its time (the bin index is taken in
// FP64 as the oracle takes it), and every particle inside the fine box adds 1
// and its velocity to the cube that holds it.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pic_internal.cuh"

namespace pic {
namespace {

__global__ void k_eepf64(const double4* __restrict__ pos, const double4* __restrict__ vel,
                         const unsigned long long* nslot, unsigned long long* hist, int nxy, int nb, double de,
                         double hm)
{
    const unsigned long long n = nslot[0];
    const int lane = threadIdx.x & 31;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const double4 p = pos[q];
        int key = -1;
        if (p.w >= 0.0) {
            const double4 v = vel[q];
            const double v2 = v.x * v.x + v.y * v.y + v.z * v.z;
            const double eps = v2 * hm;
            const double t = eps / de;
            const int b = t < (double)nb ? (int)t : nb;
            key = ((int)p.w / nxy) * (nb + 1) + b;
        }
        const unsigned m = __match_any_sync(__activemask(), key);
        if (key >= 0 && lane == __ffs(m) - 1) atomicAdd(hist + key, (unsigned long long)__popc(m));
    }
}

__global__ void k_eepf32(const float4* __restrict__ pos, const float4* __restrict__ vel,
                         const unsigned long long* nslot, unsigned long long* hist, int nb, float kbin)
{
    const unsigned long long n = nslot[0];
    const int lane = threadIdx.x & 31;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const int c = __float_as_int(pos[q].w);
        int key = -1;
        if (c >= 0) {
            const float4 v = vel[q];
            const float t = (v.x * v.x + v.y * v.y + v.z * v.z) * kbin;
            const int b = t < (float)nb ? (int)t : nb;
            key = (c >> 20) * (nb + 1) + b;
        }
        const unsigned m = __match_any_sync(__activemask(), key);
        if (key >= 0 && lane == __ffs(m) - 1) atomicAdd(hist + key, (unsigned long long)__popc(m));
    }
}

// bin = floor(frac(f_rf t + phase / 2 pi) * nph) of the sample at t = step dt
__global__ void k_phase_bin(const uint32_t* step, double f_rf, double dt, double phase, int nph, int* bin,
                            unsigned long long* bsteps)
{
    const double t = (double)*step * dt;
    const double u = f_rf * t + phase / (2.0 * 3.14159265358979323846);
    const double fr = u - floor(u);
    int b = (int)(fr * (double)nph);
    b = b < nph ? b : nph - 1;
    *bin = b;
    bsteps[b] += 1ull;
}

struct FineBox {
    double o[3], h;
    int n[3];
};

// the cube of the box holding x, or -1
__device__ __forceinline__ long long fine_cube(const FineBox& f, const double x[3])
{
    int c[3];
    for (int a = 0; a < 3; ++a) {
        const double q = (x[a] - f.o[a]) / f.h;
        if (!(q >= 0.0) || !(q < (double)f.n[a])) return -1;
        c[a] = (int)q;
    }
    return ((long long)c[2] * f.n[1] + c[1]) * f.n[0] + c[0];
}

__device__ __forceinline__ void fine_add(double* m, double vx, double vy, double vz)
{
    atomicAdd(m, 1.0);
    atomicAdd(m + 1, vx);
    atomicAdd(m + 2, vy);
    atomicAdd(m + 3, vz);
}

__global__ void k_fine64(FineBox f, const double4* __restrict__ pos, const double4* __restrict__ vel,
                         const unsigned long long* nslot, int sp, double* fine)
{
    const unsigned long long n = nslot[sp];
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const double4 p = pos[q];
        if (p.w < 0.0) continue;
        const double x[3] = {p.x, p.y, p.z};
        const long long cube = fine_cube(f, x);
        if (cube < 0) continue;
        const double4 v = vel[q];
        fine_add(fine + 4 * cube, v.x, v.y, v.z);
    }
}

// mixed layout: integer cell packed as i | j << 10 | k << 20, float offsets in
// cells, velocities in cells per step
__global__ void k_fine32(FineBox f, double dx, double vs, const float4* __restrict__ pos,
                         const float4* __restrict__ vel, const unsigned long long* nslot, int sp, double* fine)
{
    const unsigned long long n = nslot[sp];
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const float4 p = pos[q];
        const int cell = __float_as_int(p.w);
        if (cell < 0) continue;
        const double x[3] = {((double)(cell & 1023) + (double)p.x) * dx,
                             ((double)((cell >> 10) & 1023) + (double)p.y) * dx,
                             ((double)(cell >> 20) + (double)p.z) * dx};
        const long long cube = fine_cube(f, x);
        if (cube < 0) continue;
        const float4 v = vel[q];
        fine_add(fine + 4 * cube, (double)v.x * vs, (double)v.y * vs, (double)v.z * vs);
    }
}

// weighted least squares y = a + s x; false without two distinct abscissae
bool line_fit(const std::vector<double>& x, const std::vector<double>& y, const std::vector<double>& w, size_t lo,
              size_t hi, double& a, double& s)
{
    double sw = 0, sx = 0, sy = 0, sxx = 0, sxy = 0;
    for (size_t i = lo; i < hi; ++i) {
        sw += w[i]; sx += w[i] * x[i]; sy += w[i] * y[i];
        sxx += w[i] * x[i] * x[i]; sxy += w[i] * x[i] * y[i];
    }
    const double den = sw * sxx - sx * sx;
    if (hi - lo < 2 || !(den > 0.0)) return false;
    s = (sw * sxy - sx * sy) / den;
    a = (sy - s * sx) / sw;
    return true;
}

}  // namespace

void launch_eepf(pic_ctx* c)
{
    const int grid = grid_for(c->cap[0], 256, 152 * 8);
    if (c->prec == PIC_MIXED) {
        const double vs = c->dx / c->dt;
        k_eepf32<<<grid, 256, 0, c->stream>>>((const float4*)c->pos[0], (const float4*)c->vel[0], c->d_nslot,
                                              c->eepf, c->eepf_bins, (float)(vs * vs * c->hm[0] / c->eepf_de));
    } else {
        k_eepf64<<<grid, 256, 0, c->stream>>>((const double4*)c->pos[0], (const double4*)c->vel[0], c->d_nslot,
                                              c->eepf, c->nx * c->ny, c->eepf_bins, c->eepf_de, c->hm[0]);
    }
    c->launches += 1;
}

void launch_phase_bin(pic_ctx* c)
{
    k_phase_bin<<<1, 1, 0, c->stream>>>(c->d_step, c->f_rf, c->dt, c->rf_phase, c->nph, c->d_bin, c->d_bsteps);
    c->launches += 1;
}

void launch_fine(pic_ctx* c)
{
    FineBox f;
    for (int a = 0; a < 3; ++a) { f.o[a] = c->fine_o[a]; f.n[a] = c->fine_n[a]; }
    f.h = c->fine_h;
    for (int sp = 0; sp < 2; ++sp) {
        const int grid = grid_for(c->cap[sp], 256, 152 * 8);
        if (c->prec == PIC_MIXED)
            k_fine32<<<grid, 256, 0, c->stream>>>(f, c->dx, c->dx / c->dt, (const float4*)c->pos[sp],
                                                  (const float4*)c->vel[sp], c->d_nslot, sp, c->fine[sp]);
        else
            k_fine64<<<grid, 256, 0, c->stream>>>(f, (const double4*)c->pos[sp], (const double4*)c->vel[sp],
                                                  c->d_nslot, sp, c->fine[sp]);
    }
    c->launches += 2;
}

}  // namespace pic

extern "C" {

// Two-Maxwellian fit of g(eps) = counts_b / (de sqrt(eps_b)) at the bin centres
// eps_b = (b + 1/2) de in [e_lo, e_hi]: g = A_l exp(-eps/T_l) + A_h exp(-eps/T_h).
// The hot group is a weighted line fit of ln g over the bins from a split on,
// the cold group a line fit of ln(g - hot part) below it; the split with the
// least weighted squared log residual over all bins wins (weights = counts, the
// inverse variance of ln g for Poisson counts).
pic_status pic_eepf_fit(const int64_t* counts, int32_t nbins, double de_ev, double e_lo_ev, double e_hi_ev,
                        double* fit)
{
    if (!counts || !fit || nbins < 4 || !(de_ev > 0.0) || !(e_hi_ev > e_lo_ev)) return PIC_EINVAL;
    std::vector<double> x, y, w, g;
    for (int b = 0; b < nbins; ++b) {
        const double e = (b + 0.5) * de_ev;
        if (e < e_lo_ev || e > e_hi_ev || counts[b] <= 0) continue;
        const double gv = (double)counts[b] / (de_ev * std::sqrt(e));
        x.push_back(e);
        g.push_back(gv);
        y.push_back(std::log(gv));
        w.push_back((double)counts[b]);
    }
    const size_t n = x.size();
    if (n < 4) return PIC_EINVAL;
    double best = INFINITY, out[4] = {0, 0, 0, 0};
    // one Maxwellian over everything as the fallback
    {
        double a, s;
        if (pic::line_fit(x, y, w, 0, n, a, s) && s < 0.0) {
            double cost = 0;
            for (size_t i = 0; i < n; ++i) cost += w[i] * (a + s * x[i] - y[i]) * (a + s * x[i] - y[i]);
            best = cost;
            out[0] = out[1] = -1.0 / s;
            out[2] = 0.0;
            out[3] = std::exp(a);
        }
    }
    for (size_t split = 2; split + 2 <= n; ++split) {
        double ah, sh;
        if (!pic::line_fit(x, y, w, split, n, ah, sh) || !(sh < 0.0)) continue;
        std::vector<double> yl(split), wl(split);
        bool ok = true;
        for (size_t i = 0; i < split; ++i) {
            const double r = g[i] - std::exp(ah + sh * x[i]);
            if (!(r > 0.0)) { ok = false; break; }
            yl[i] = std::log(r);
            wl[i] = w[i] * (r / g[i]) * (r / g[i]);
        }
        if (!ok) continue;
        double al, sl;
        if (!pic::line_fit(x, yl, wl, 0, split, al, sl) || !(sl < sh)) continue;
        double cost = 0;
        for (size_t i = 0; i < n; ++i) {
            const double m = std::log(std::exp(al + sl * x[i]) + std::exp(ah + sh * x[i]));
            cost += w[i] * (m - y[i]) * (m - y[i]);
        }
        if (cost < best) {
            best = cost;
            out[0] = -1.0 / sl;
            out[1] = -1.0 / sh;
            out[2] = std::exp(al);
            out[3] = std::exp(ah);
        }
    }
    if (!(best < INFINITY)) return PIC_EINVAL;
    for (int i = 0; i < 4; ++i) fit[i] = out[i];
    return PIC_OK;
}

}  // extern "C"

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

// Hypothetical charge of each grain with no other grains around (Sec. IV.B):
// the orbital-motion-limited balance of electron and ion currents with the
// charge-exchange ion current, from the local moments.  Currents per pi a^2,
// mean speeds vbar = sqrt(8 e T / (pi m)), x = phi / T_i:
//   phi <= 0: J_e = n_e vbar_e exp(phi/T_e),  J_i = n_i vbar_i (1 - x + 0.1 x^2 lambda_D / l_i)
//   phi >  0: J_e = n_e vbar_e (1 + phi/T_e), J_i = n_i vbar_i exp(-x)
// (the quadratic term: weakly collisional charge exchange, Khrapak et al.,
// Phys. Rev. E 72, 016406 (2005)); lambda_D = (lambda_De^-2 + lambda_Di^-2)^-1/2,
// l_i = 1 / (n_gas sigma_cx(3/2 T_i)).  The local n, <v>, <v^2> are the
// window sums CIC-interpolated to the grain centre; phi solves J_e = J_i by a
// bracketed Newton iteration; Q = 4 pi eps0 a phi.
struct OmlArgs {
    const double* mom[2];
    const double* mke[2];
    const double* gpos;
    const double* grad;
    const double* xs_cx;
    int n_xs, ng, nph, nx, ny, nz;
    size_t nodes;
    double dx, norm, de_i, n_gas, m3e[2];
    int with_cx;
};

// J_e - J_i over n_i vbar_i and its derivative in phi
__device__ void oml_balance(double phi, double A, double te, double ti, double lam_l, double& f, double& df)
{
    if (phi <= 0.0) {
        const double x = phi / ti;
        const double ee = A * exp(phi / te);
        f = ee - (1.0 - x + 0.1 * x * x * lam_l);
        df = ee / te + (1.0 - 0.2 * x * lam_l) / ti;
    } else {
        const double ei = exp(-phi / ti);
        f = A * (1.0 + phi / te) - ei;
        df = A / te + ei / ti;
    }
}

__global__ void k_oml(OmlArgs a, double* out)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.ng) return;
    const double p[3] = {a.gpos[3 * g], a.gpos[3 * g + 1], a.gpos[3 * g + 2]};
    const int nn[3] = {a.nx, a.ny, a.nz};
    int c[3];
    double f[3];
    for (int d = 0; d < 3; ++d) {
        const double q = p[d] / a.dx;
        int i = (int)floor(q);
        i = i > nn[d] - 1 ? nn[d] - 1 : (i < 0 ? 0 : i);
        c[d] = i;
        f[d] = q - (double)i;
    }
    double s[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int di = 0; di < 2; ++di) {
                const double w = (di ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                const int i = (c[0] + di) % a.nx, j = (c[1] + dy) % a.ny, k = c[2] + dz;
                const size_t node = ((size_t)k * a.ny + j) * a.nx + i;
                for (int sp = 0; sp < 2; ++sp) {
                    double t[5] = {0, 0, 0, 0, 0};
                    for (int b = 0; b < a.nph; ++b) {
                        const double* m = a.mom[sp] + 4 * ((size_t)b * a.nodes + node);
                        t[0] += m[0]; t[1] += m[1]; t[2] += m[2]; t[3] += m[3];
                        t[4] += a.mke[sp][(size_t)b * a.nodes + node];
                    }
                    for (int q = 0; q < 5; ++q) s[sp][q] += w * t[q];
                }
            }
    double n[2], T[2];
    for (int sp = 0; sp < 2; ++sp) {
        n[sp] = s[sp][0] * a.norm;
        if (s[sp][0] > 0.0) {
            const double u0 = s[sp][1] / s[sp][0], u1 = s[sp][2] / s[sp][0], u2 = s[sp][3] / s[sp][0];
            T[sp] = a.m3e[sp] * (s[sp][4] / s[sp][0] - ((u0 * u0 + u1 * u1) + u2 * u2));
        } else {
            T[sp] = 0.0;
        }
    }
    double phi = nan("");
    if (n[0] > 0.0 && n[1] > 0.0 && T[0] > 0.0 && T[1] > 0.0) {
        double lam_l = 0.0;
        if (a.with_cx && a.n_xs > 1) {
            const double lde2 = (kEPS0 * T[0]) / (n[0] * kQE), ldi2 = (kEPS0 * T[1]) / (n[1] * kQE);
            const double lam = 1.0 / sqrt(1.0 / lde2 + 1.0 / ldi2);
            const double t = (1.5 * T[1]) / a.de_i;
            double sig;
            if (t >= (double)(a.n_xs - 1)) {
                sig = a.xs_cx[a.n_xs - 1];
            } else {
                const int i = (int)t;
                sig = a.xs_cx[i] + (t - (double)i) * (a.xs_cx[i + 1] - a.xs_cx[i]);
            }
            lam_l = lam * (a.n_gas * sig);
        }
        const double ve = sqrt((8.0 * kQE * T[0]) / (kPI * kME));
        const double vi = sqrt((8.0 * kQE * T[1]) / (kPI * kMAR));
        const double A = (n[0] * ve) / (n[1] * vi);
        double lo = A > 1.0 ? -200.0 * T[0] : 0.0, hi = A > 1.0 ? 0.0 : 200.0 * T[1];
        phi = A == 1.0 ? 0.0 : 0.5 * (lo + hi);
        for (int it = 0; it < 200 && A != 1.0; ++it) {
            double fv, dfv;
            oml_balance(phi, A, T[0], T[1], lam_l, fv, dfv);
            if (fv > 0.0) hi = phi; else lo = phi;
            double nxt = phi - fv / dfv;
            if (!(nxt > lo && nxt < hi)) nxt = 0.5 * (lo + hi);   // outside the bracket: bisect
            if (nxt == phi || hi - lo <= 4e-16 * fmax(fabs(lo), fabs(hi))) { phi = nxt; break; }
            phi = nxt;
        }
    }
    double* o = out + 6 * g;
    o[0] = 4.0 * kPI * kEPS0 * a.grad[g] * phi;
    o[1] = phi;
    o[2] = n[0]; o[3] = n[1]; o[4] = T[0]; o[5] = T[1];
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

void launch_oml(pic_ctx* c, int with_cx, double* out)
{
    OmlArgs a;
    for (int sp = 0; sp < 2; ++sp) {
        a.mom[sp] = c->mom[sp];
        a.mke[sp] = c->mke[sp];
        a.m3e[sp] = (2.0 / 3.0) * c->hm[sp];
    }
    a.gpos = c->gpos; a.grad = c->grad; a.xs_cx = c->xs64 + 4 * (size_t)c->n_xs;
    a.n_xs = c->n_xs; a.ng = c->ng; a.nph = c->nph; a.nx = c->nx; a.ny = c->ny; a.nz = c->nz;
    a.nodes = c->nodes; a.dx = c->dx;
    a.norm = c->W / ((c->dx * c->dx * c->dx) * (double)c->msteps);
    a.de_i = c->de[1]; a.n_gas = c->n_gas; a.with_cx = with_cx;
    k_oml<<<(c->ng + 127) / 128, 128, 0, c->stream>>>(a, out);
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

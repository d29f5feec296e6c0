// FP64 particle cycle (Sec. III): CIC gather of the finite-difference field
// (Eqs. 3-4), leapfrog push (Eqs. 1-2), MD subcycling with the PPPM
// correction near grains (Eqs. 5-6), grain and electrode absorption,
// null-collision MCC with the argon background (Table I) and the fixed-point
// CIC deposit.
//
// This translation unit is compiled with --fmad=false: every product and sum
// rounds on its own, in the order written, so an FP64 step on the GPU is
// bit-identical to a plain FP64 CPU evaluation of the same formulas.
#include "pic_internal.cuh"

namespace pic {
namespace {

struct P64 {
    int nx, ny, nz;
    double dx, Lx, Ly, Lz;
    double dt, dtm;
    int M;
    int sp;
    double qmdt, qmdtm, hm, pnull, nu_max, de;
    double n_gas, sig_n, eps_exc, eps_ion, mr2, kc;
    int n_xs;
    const double* xs;
    uint2 key;
    const uint32_t* step;        // device step counter (Philox counter word 2)
    int flags;
    int ng;
    const double* gpos;
    const double* grad;
    const int* gcell;
    const double* gq;
    const double* gtab;
    unsigned long long* gabs;
    const int* cell_ng;
    const int* cell_g;
    const double* ex;
    const double* ey;
    const double* ez;
    unsigned long long* rq;
    double4* pos;
    double4* vel;
    const unsigned long long* nslot;
    unsigned long long* cnt;
    int* err;
    ChildRec* child;
    unsigned long long child_cap;
    unsigned long long* nch;
};

struct Geo {
    int nx, ny, nz;
    double dx, Lx, Ly, Lz;
};

__device__ __forceinline__ void locate(const Geo& g, const double x[3], int c[3], double f[3])
{
    const int nn[3] = {g.nx, g.ny, g.nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double q = x[a] / g.dx;
        int i = (int)floor(q);
        if (i > nn[a] - 1) i = nn[a] - 1;
        if (i < 0) i = 0;
        c[a] = i;
        f[a] = q - (double)i;
    }
}

__device__ __forceinline__ void qweights(const double f[3], long long w[3][2])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        long long q = (long long)rint(f[a] * (double)kWQ);
        if (q < 0) q = 0;
        if (q > kWQ) q = kWQ;
        w[a][0] = kWQ - q;
        w[a][1] = q;
    }
}

__device__ __forceinline__ size_t node_at(const Geo& g, int i, int j, int k)
{
    i %= g.nx;
    j %= g.ny;
    return ((size_t)k * g.ny + j) * g.nx + i;
}

__device__ __forceinline__ int cell_of(const Geo& g, const int c[3]) { return (c[2] * g.ny + c[1]) * g.nx + c[0]; }

__device__ __forceinline__ void deposit(const Geo& g, unsigned long long* rq, const int c[3], const long long w[3][2],
                                        long long charge)
{
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int di = 0; di < 2; ++di) {
                const long long v = charge * (w[0][di] * w[1][dy] * w[2][dz]);
                if (v != 0) atomicAdd(rq + node_at(g, c[0] + di, c[1] + dy, c[2] + dz), (unsigned long long)v);
            }
}

__device__ __forceinline__ void gather(const Geo& g, const double* fx, const double* fy, const double* fz,
                                       const int c[3], const long long w[3][2], double E[3])
{
    E[0] = 0.0; E[1] = 0.0; E[2] = 0.0;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int di = 0; di < 2; ++di) {
                const double wt = (double)(w[0][di] * w[1][dy] * w[2][dz]) * 0x1p-42;
                const size_t n = node_at(g, c[0] + di, c[1] + dy, c[2] + dz);
                E[0] = E[0] + wt * fx[n];
                E[1] = E[1] + wt * fy[n];
                E[2] = E[2] + wt * fz[n];
            }
}

__device__ __forceinline__ void grain_sep(const P64& p, int gi, const double x[3], double d[3])
{
    const double L[2] = {p.Lx, p.Ly};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        double q = x[a] - p.gpos[3 * gi + a];
        if (q > 0.5 * L[a]) q = q - L[a];
        else if (q < -0.5 * L[a]) q = q + L[a];
        d[a] = q;
    }
    d[2] = x[2] - p.gpos[3 * gi + 2];
}

// E = E_PIC - Q g(x) + Q (x - x_g) / (4 pi eps0 |x - x_g|^3) for the grains whose
// MD region holds the particle's cell (Eqs. 5-6)
__device__ void md_correct(const P64& p, const Geo& g, const double x[3], const int c[3], const long long w[3][2],
                           double E[3])
{
    const int cell = cell_of(g, c);
    const int n = p.cell_ng[cell];
    for (int t = 0; t < n; ++t) {
        const int gi = p.cell_g[cell * kMaxG + t];
        const int gc0 = p.gcell[3 * gi], gc1 = p.gcell[3 * gi + 1], gc2 = p.gcell[3 * gi + 2];
        double Ed[3] = {0.0, 0.0, 0.0};
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int di = 0; di < 2; ++di) {
                    const double wt = (double)(w[0][di] * w[1][dy] * w[2][dz]) * 0x1p-42;
                    const int li = ((c[0] + di - gc0 + 1) % g.nx + g.nx) % g.nx;
                    const int lj = ((c[1] + dy - gc1 + 1) % g.ny + g.ny) % g.ny;
                    const int lk = c[2] + dz - gc2 + 1;
                    const double* tv = p.gtab + ((size_t)gi * 64 + (lk * 4 + lj) * 4 + li) * 3;
                    Ed[0] = Ed[0] + wt * tv[0];
                    Ed[1] = Ed[1] + wt * tv[1];
                    Ed[2] = Ed[2] + wt * tv[2];
                }
        double d[3];
        grain_sep(p, gi, x, d);
        const double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        const double Q = p.gq[gi];
        double coef = 0.0;
        if (r2 > 0.0) {
            const double r = sqrt(r2);
            coef = (Q * p.kc) / (r2 * r);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) E[a] = (E[a] - Q * Ed[a]) + coef * d[a];
    }
}

// 0 alive, 1 lost at z = 0, 2 lost at z = Lz, 3 invalid
__device__ __forceinline__ int boundary(const Geo& g, double x[3])
{
    if (!(x[2] >= 0.0)) return (x[2] < 0.0) ? 1 : 3;
    if (x[2] > g.Lz) return 2;
    const double L[2] = {g.Lx, g.Ly};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        if (x[a] < 0.0) x[a] = x[a] + L[a];
        else if (x[a] >= L[a]) x[a] = x[a] - L[a];
        if (!(x[a] >= 0.0 && x[a] <= L[a])) return 3;
    }
    return 0;
}

__device__ int absorbed_by(const P64& p, const Geo& g, const double x[3])
{
    int c[3];
    double f[3];
    locate(g, x, c, f);
    const int cell = cell_of(g, c);
    const int n = p.cell_ng[cell];
    for (int t = 0; t < n; ++t) {
        const int gi = p.cell_g[cell * kMaxG + t];
        double d[3];
        grain_sep(p, gi, x, d);
        const double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        if (r2 <= p.grad[gi] * p.grad[gi]) return gi;
    }
    return -1;
}

__device__ __forceinline__ double xs_at(const double* tab, int n, double de, double eps)
{
    const double t = eps / de;
    if (t >= (double)(n - 1)) return tab[n - 1];
    const int i = (int)t;
    const double fr = t - (double)i;
    return tab[i] + fr * (tab[i + 1] - tab[i]);
}

__device__ __forceinline__ void pair(RStream& r, double& a, double& b)
{
    const uint32_t ua = r.next(), ub = r.next();
    a = 2.0 * u01d(ua) - 1.0;
    b = 2.0 * u01d(ub) - 1.0;
}

// isotropic direction (Marsaglia 1972)
__device__ void iso(RStream& r, double o[3])
{
    for (int t = 0; t < 128; ++t) {
        double a, b;
        pair(r, a, b);
        const double s = a * a + b * b;
        if (s < 1.0) {
            const double q = 2.0 * sqrt(1.0 - s);
            o[0] = a * q; o[1] = b * q; o[2] = 1.0 - 2.0 * s;
            return;
        }
    }
    o[0] = 0.0; o[1] = 0.0; o[2] = 1.0;
}

// two standard normals (Marsaglia polar method)
__device__ void gauss2(RStream& r, double& n1, double& n2)
{
    for (int t = 0; t < 128; ++t) {
        double a, b;
        pair(r, a, b);
        const double s = a * a + b * b;
        if (s < 1.0) {
            const double f = sqrt((-2.0 * ln_series(s)) / s);
            n1 = a * f; n2 = b * f;
            return;
        }
    }
    n1 = 0.0; n2 = 0.0;
}

__device__ void gauss3(RStream& r, double o[3])
{
    double d;
    gauss2(r, o[0], o[1]);
    gauss2(r, o[2], d);
}

__device__ __forceinline__ void latch(int* err, int code) { atomicCAS(err, 0, code); }

// null-collision MCC after the push (Table I); may record an ionization product
__device__ void mcc(const P64& p, uint32_t step, const double x[3], double v[3], uint32_t id, int cell)
{
    const uint4 u = philox4x32_10(make_uint4(id, step, kPurMCC, 0u), p.key);
    if (u01d(u.x) >= p.pnull) return;
    const double ng = p.n_gas;
    const int nx = p.n_xs;
    if (p.sp == 0) {
        const double v2 = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
        const double eps = v2 * p.hm;
        const double vm = sqrt(v2);
        const double nu_el = (ng * xs_at(p.xs + 0 * nx, nx, p.de, eps)) * vm;
        const double nu_ex = (ng * xs_at(p.xs + 1 * nx, nx, p.de, eps)) * vm;
        const double nu_io = (ng * xs_at(p.xs + 2 * nx, nx, p.de, eps)) * vm;
        const double R = u01d(u.y) * p.nu_max;
        double acc = nu_el;
        RStream rd(id, step, kPurDir, p.key);
        double dir[3];
        if (R < acc) {
            iso(rd, dir);
            const double cosx = ((dir[0] * v[0] + dir[1] * v[1]) + dir[2] * v[2]) / vm;
            const double fac = 1.0 - p.mr2 * (1.0 - cosx);
            const double vn = vm * sqrt(fac);
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a] = vn * dir[a];
            atomicAdd(p.cnt + PIC_C_E_EL, 1ull);
            return;
        }
        acc = acc + nu_ex;
        if (R < acc) {
            double e2 = eps - p.eps_exc;
            if (e2 < 0.0) e2 = 0.0;
            iso(rd, dir);
            const double vn = sqrt(e2 / p.hm);
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a] = vn * dir[a];
            atomicAdd(p.cnt + PIC_C_E_EXC, 1ull);
            return;
        }
        acc = acc + nu_io;
        if (R < acc) {
            double e2 = eps - p.eps_ion;
            if (e2 < 0.0) e2 = 0.0;
            const double vn = sqrt((0.5 * e2) / p.hm);
            iso(rd, dir);
            ChildRec cr;
            cr.parent = id;
            cr.cell = cell;
#pragma unroll
            for (int a = 0; a < 3; ++a) { v[a] = vn * dir[a]; cr.x[a] = x[a]; }
            double d2[3], gn[3];
            RStream rc(id, step, kPurChildDir, p.key);
            iso(rc, d2);
            RStream rn(id, step, kPurChildNeutral, p.key);
            gauss3(rn, gn);
#pragma unroll
            for (int a = 0; a < 3; ++a) { cr.ve[a] = vn * d2[a]; cr.vi[a] = p.sig_n * gn[a]; }
            const unsigned long long slot = atomicAdd(p.nch, 1ull);
            if (slot < p.child_cap) p.child[slot] = cr;
            else latch(p.err, kErrCapacity);
            atomicAdd(p.cnt + PIC_C_E_ION, 1ull);
        }
        return;
    }
    double gn[3];
    RStream rn(id, step, kPurNeutral, p.key);
    gauss3(rn, gn);
    const double vn[3] = {p.sig_n * gn[0], p.sig_n * gn[1], p.sig_n * gn[2]};
    const double gv[3] = {v[0] - vn[0], v[1] - vn[1], v[2] - vn[2]};
    const double g2 = (gv[0] * gv[0] + gv[1] * gv[1]) + gv[2] * gv[2];
    const double eps = g2 * p.hm;
    const double gm = sqrt(g2);
    const double nu_el = (ng * xs_at(p.xs + 3 * nx, nx, p.de, eps)) * gm;
    const double nu_cx = (ng * xs_at(p.xs + 4 * nx, nx, p.de, eps)) * gm;
    const double R = u01d(u.y) * p.nu_max;
    double acc = nu_el;
    if (R < acc) {
        double dir[3];
        RStream rd(id, step, kPurDir, p.key);
        iso(rd, dir);
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = (v[a] + vn[a]) * 0.5 + (0.5 * gm) * dir[a];
        atomicAdd(p.cnt + PIC_C_I_EL, 1ull);
        return;
    }
    acc = acc + nu_cx;
    if (R < acc) {
#pragma unroll
        for (int a = 0; a < 3; ++a) v[a] = vn[a];
        atomicAdd(p.cnt + PIC_C_I_CX, 1ull);
    }
}

__global__ void k_push64(const P64 p)
{
    const Geo g{p.nx, p.ny, p.nz, p.dx, p.Lx, p.Ly, p.Lz};
    const unsigned long long n = p.nslot[p.sp];
    const uint32_t step = *p.step;
    const bool frozen = (p.sp == 1) && (p.flags & PIC_F_IONS_FROZEN);
    const long long charge = p.sp == 0 ? -1 : 1;
    unsigned int live = 0;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        double4 P = p.pos[q];
        if (P.w < 0.0) continue;
        ++live;
        double x[3] = {P.x, P.y, P.z};
        int c[3];
        double f[3];
        long long w[3][2];
        if (frozen) {
            locate(g, x, c, f);
            qweights(f, w);
            deposit(g, p.rq, c, w, charge);
            continue;
        }
        const double4 V = p.vel[q];
        double v[3] = {V.x, V.y, V.z};
        const uint32_t id = (uint32_t)V.w;
        locate(g, x, c, f);
        qweights(f, w);
        int fate = 0, grain = -1;
        if (p.cell_ng[cell_of(g, c)] == 0) {
            double E[3];
            gather(g, p.ex, p.ey, p.ez, c, w, E);
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a] = v[a] + p.qmdt * E[a];
#pragma unroll
            for (int a = 0; a < 3; ++a) x[a] = x[a] + v[a] * p.dt;
            fate = boundary(g, x);
        } else {
            for (int m = 0; m < p.M; ++m) {
                double E[3];
                if (m > 0) {
                    locate(g, x, c, f);
                    qweights(f, w);
                }
                gather(g, p.ex, p.ey, p.ez, c, w, E);
                md_correct(p, g, x, c, w, E);
#pragma unroll
                for (int a = 0; a < 3; ++a) v[a] = v[a] + p.qmdtm * E[a];
#pragma unroll
                for (int a = 0; a < 3; ++a) x[a] = x[a] + v[a] * p.dtm;
                fate = boundary(g, x);
                if (fate) break;
                grain = absorbed_by(p, g, x);
                if (grain >= 0) break;
            }
        }
        if (fate != 0 || grain >= 0) {
            p.pos[q].w = -1.0;
            if (fate == 1) atomicAdd(p.cnt + (p.sp == 0 ? PIC_C_LOST_BOT_E : PIC_C_LOST_BOT_I), 1ull);
            else if (fate == 2) atomicAdd(p.cnt + (p.sp == 0 ? PIC_C_LOST_TOP_E : PIC_C_LOST_TOP_I), 1ull);
            else if (fate == 3) {
                atomicAdd(p.cnt + PIC_C_ERR, 1ull);
                latch(p.err, kErrNonFinite);
            } else {
                atomicAdd(p.gabs + 2 * grain + p.sp, 1ull);
                atomicAdd(p.cnt + (p.sp == 0 ? PIC_C_ABS_E : PIC_C_ABS_I), 1ull);
            }
            continue;
        }
        locate(g, x, c, f);
        const int cell = cell_of(g, c);
        if (!(p.flags & PIC_F_NO_MCC)) mcc(p, step, x, v, id, cell);
        p.pos[q] = make_double4(x[0], x[1], x[2], (double)cell);
        p.vel[q] = make_double4(v[0], v[1], v[2], (double)id);
        qweights(f, w);
        deposit(g, p.rq, c, w, charge);
    }
    live = __reduce_add_sync(0xffffffffu, live);
    if ((threadIdx.x & 31) == 0 && live) atomicAdd(p.cnt + PIC_C_PUSHED, (unsigned long long)live);
}

// deposit every live particle (initial rho and re-deposits)
__global__ void k_deposit64(Geo g, const double4* pos, const unsigned long long* nslot, int sp,
                            unsigned long long* rq)
{
    const unsigned long long n = nslot[sp];
    const long long charge = sp == 0 ? -1 : 1;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const double4 P = pos[q];
        if (P.w < 0.0) continue;
        const double x[3] = {P.x, P.y, P.z};
        int c[3];
        double f[3];
        long long w[3][2];
        locate(g, x, c, f);
        qweights(f, w);
        deposit(g, rq, c, w, charge);
    }
}

// E = -grad phi at the nodes (Eq. 4): central differences, one-sided second
// order on the electrode planes
__global__ void k_efield64(int nx, int ny, int nz, double dx, const double* __restrict__ phi, double* __restrict__ ex,
                           double* __restrict__ ey, double* __restrict__ ez)
{
    const size_t P = (size_t)nx * ny;
    const size_t N = P * (nz + 1);
    const double h2 = 2.0 * dx;
    for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(n % nx);
        const int j = (int)((n / nx) % ny);
        const int k = (int)(n / P);
        const size_t row = ((size_t)k * ny + j) * nx;
        const int ip = (i + 1) % nx, im = (i + nx - 1) % nx;
        const int jp = (j + 1) % ny, jm = (j + ny - 1) % ny;
        ex[n] = (phi[row + im] - phi[row + ip]) / h2;
        ey[n] = (phi[((size_t)k * ny + jm) * nx + i] - phi[((size_t)k * ny + jp) * nx + i]) / h2;
        if (k == 0)
            ez[n] = ((3.0 * phi[n] - 4.0 * phi[n + P]) + phi[n + 2 * P]) / h2;
        else if (k == nz)
            ez[n] = ((4.0 * phi[n - P] - 3.0 * phi[n]) - phi[n - 2 * P]) / h2;
        else
            ez[n] = (phi[n - P] - phi[n + P]) / h2;
    }
}

// Number the ionization products by their parents' ids (rank among this
// step's parents), append electron/ion pairs after the live slots, deposit.
__global__ void k_children64(Geo g, ChildRec* rec, const unsigned long long* nch, unsigned long long child_cap,
                             const unsigned long long* nslot, const unsigned int* next_id, double4* pos_e,
                             double4* vel_e, double4* pos_i, double4* vel_i, long long cap_e, long long cap_i,
                             unsigned long long* rq, int* err)
{
    __shared__ uint32_t tile[256];
    const unsigned long long n = min(*nch, child_cap);   // records past the buffer were never written
    const unsigned long long base_e = nslot[0], base_i = nslot[1];
    const unsigned int nid = *next_id;
    for (unsigned long long r0 = blockIdx.x * (unsigned long long)blockDim.x; r0 < n;
         r0 += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long r = r0 + threadIdx.x;
        const uint32_t mine = r < n ? rec[r].parent : 0xFFFFFFFFu;
        unsigned long long rank = 0;
        for (unsigned long long t0 = 0; t0 < n; t0 += blockDim.x) {
            __syncthreads();
            tile[threadIdx.x] = (t0 + threadIdx.x < n) ? rec[t0 + threadIdx.x].parent : 0xFFFFFFFFu;
            __syncthreads();
            const int lim = (int)min((unsigned long long)blockDim.x, n - t0);
            for (int t = 0; t < lim; ++t) rank += tile[t] < mine;
        }
        if (r >= n) continue;
        const ChildRec cr = rec[r];
        const unsigned long long se = base_e + rank, si = base_i + rank;
        if (se >= (unsigned long long)cap_e || si >= (unsigned long long)cap_i) {
            atomicCAS(err, 0, (int)kErrCapacity);
            continue;
        }
        const double x[3] = {cr.x[0], cr.x[1], cr.x[2]};
        int c[3];
        double f[3];
        long long w[3][2];
        locate(g, x, c, f);
        qweights(f, w);
        const double cell = (double)cell_of(g, c);
        pos_e[se] = make_double4(x[0], x[1], x[2], cell);
        vel_e[se] = make_double4(cr.ve[0], cr.ve[1], cr.ve[2], (double)(nid + (unsigned)(2 * rank)));
        pos_i[si] = make_double4(x[0], x[1], x[2], cell);
        vel_i[si] = make_double4(cr.vi[0], cr.vi[1], cr.vi[2], (double)(nid + (unsigned)(2 * rank + 1)));
        deposit(g, rq, c, w, -1);
        deposit(g, rq, c, w, 1);
    }
}

__global__ void k_children_finish(unsigned long long* nch, unsigned long long child_cap, unsigned long long* nslot,
                                  unsigned int* next_id, long long cap_e, long long cap_i, uint32_t* step)
{
    *step += 1u;   // the step is complete on the particle side
    const unsigned long long n = min(*nch, child_cap);
    nslot[0] = min(nslot[0] + n, (unsigned long long)cap_e);
    nslot[1] = min(nslot[1] + n, (unsigned long long)cap_i);
    *next_id += (unsigned int)(2 * n);
    *nch = 0;
}

// grain charges from the exact counts (Q = e W (N_ion - N_e)) and their CIC deposit
__global__ void k_grains(Geo g, int ng, double qw, const unsigned long long* gabs, const double* gpos, double* gq,
                         float* gq32, unsigned long long* rq)
{
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ng) return;
    const long long net = (long long)gabs[2 * gi + 1] - (long long)gabs[2 * gi];
    const double Q = qw * (double)net;
    gq[gi] = Q;
    gq32[gi] = (float)Q;
    const double x[3] = {gpos[3 * gi], gpos[3 * gi + 1], gpos[3 * gi + 2]};
    int c[3];
    double f[3];
    long long w[3][2];
    locate(g, x, c, f);
    qweights(f, w);
    deposit(g, rq, c, w, net);
}

// E of the current phi on the 4x4x4 nodes of grain gi's region (unit-charge table)
__global__ void k_grain_table(int nx, int ny, int nz, double dx, const double* phi, const int* gcell, int gi,
                              double* tab)
{
    const int t = threadIdx.x;
    if (t >= 64) return;
    const int li = t % 4, lj = (t / 4) % 4, lk = t / 16;
    const int i = ((gcell[3 * gi] - 1 + li) % nx + nx) % nx;
    const int j = ((gcell[3 * gi + 1] - 1 + lj) % ny + ny) % ny;
    const int k = gcell[3 * gi + 2] - 1 + lk;
    const size_t P = (size_t)nx * ny;
    const size_t n = (size_t)k * P + (size_t)j * nx + i;
    const double h2 = 2.0 * dx;
    const size_t row = (size_t)k * P + (size_t)j * nx;
    double* o = tab + ((size_t)gi * 64 + t) * 3;
    o[0] = (phi[row + (i + nx - 1) % nx] - phi[row + (i + 1) % nx]) / h2;
    o[1] = (phi[(size_t)k * P + (size_t)((j + ny - 1) % ny) * nx + i] -
            phi[(size_t)k * P + (size_t)((j + 1) % ny) * nx + i]) / h2;
    if (k == 0)
        o[2] = ((3.0 * phi[n] - 4.0 * phi[n + P]) + phi[n + 2 * P]) / h2;
    else if (k == nz)
        o[2] = ((4.0 * phi[n - P] - 3.0 * phi[n]) - phi[n - 2 * P]) / h2;
    else
        o[2] = (phi[n - P] - phi[n + P]) / h2;
}

// The unit-charge tables by superposition: the mesh is periodic in x and y,
// so the potential of a unit charge on node (i, j, k) is that of a unit charge
// on node (0, 0, k) moved by (i, j).  One solve per node plane k that some
// grain's cell corners lie on gives the potential of a unit charge at (0, 0, k);
// k_green_block keeps its values at offsets -3..3 in x, y and z around that
// node.  A grain's unit charge is its CIC deposit on the 8 corners of its cell
// (the weights of k_grains, summing to 2^42), so its potential near the grain
// is the weighted sum of the 8 corners' moved blocks, and k_grain_table_sup
// takes its table from that sum with the differences of k_grain_table.
constexpr int kGreenR = 3, kGreenW = 2 * kGreenR + 1;

__global__ void k_green_block(int nx, int ny, int nz, const double* phi, int k, double* blk)
{
    const int t = threadIdx.x;
    if (t >= kGreenW * kGreenW * kGreenW) return;
    const int dx = t % kGreenW - kGreenR, dy = (t / kGreenW) % kGreenW - kGreenR, dz = t / (kGreenW * kGreenW) - kGreenR;
    const int kk = k + dz;
    double v = 0.0;
    if (kk >= 0 && kk <= nz) {
        const int i = (dx % nx + nx) % nx, j = (dy % ny + ny) % ny;
        v = phi[((size_t)kk * ny + j) * nx + i];
    }
    blk[t] = v;
}

__device__ __forceinline__ int wrap_off(int d, int n)
{
    if (2 * d > n) d -= n;
    if (2 * d < -n) d += n;
    return d;
}

// potential of grain gi's unit charge at node (i, j, k) (i, j already wrapped)
__device__ double sup_phi(const Geo& g, const double* blk, const int* plane, const int c[3], const long long w[3][2],
                          int i, int j, int k)
{
    double s = 0.0;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int di = 0; di < 2; ++di) {
                const int ci = (c[0] + di) % g.nx, cj = (c[1] + dy) % g.ny, ck = c[2] + dz;
                const int ox = wrap_off(i - ci, g.nx), oy = wrap_off(j - cj, g.ny), oz = k - ck;
                const double wt = (double)(w[0][di] * w[1][dy] * w[2][dz]) * 0x1p-42;
                const double* b = blk + (size_t)plane[ck] * (kGreenW * kGreenW * kGreenW);
                s = s + wt * b[((oz + kGreenR) * kGreenW + (oy + kGreenR)) * kGreenW + (ox + kGreenR)];
            }
    return s;
}

__global__ void k_grain_table_sup(Geo g, const double* gpos, const int* gcell, const double* blk, const int* plane,
                                  double* tab)
{
    const int gi = blockIdx.x, t = threadIdx.x;
    if (t >= 64) return;
    const double x[3] = {gpos[3 * gi], gpos[3 * gi + 1], gpos[3 * gi + 2]};
    int c[3];
    double f[3];
    long long w[3][2];
    locate(g, x, c, f);
    qweights(f, w);
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int li = t % 4, lj = (t / 4) % 4, lk = t / 16;
    const int i = ((gcell[3 * gi] - 1 + li) % nx + nx) % nx;
    const int j = ((gcell[3 * gi + 1] - 1 + lj) % ny + ny) % ny;
    const int k = gcell[3 * gi + 2] - 1 + lk;
    const double h2 = 2.0 * g.dx;
    auto ph = [&](int a, int b, int z) { return sup_phi(g, blk, plane, c, w, a, b, z); };
    double* o = tab + ((size_t)gi * 64 + t) * 3;
    o[0] = (ph((i + nx - 1) % nx, j, k) - ph((i + 1) % nx, j, k)) / h2;
    o[1] = (ph(i, (j + ny - 1) % ny, k) - ph(i, (j + 1) % ny, k)) / h2;
    if (k == 0)
        o[2] = ((3.0 * ph(i, j, k) - 4.0 * ph(i, j, k + 1)) + ph(i, j, k + 2)) / h2;
    else if (k == nz)
        o[2] = ((4.0 * ph(i, j, k - 1) - 3.0 * ph(i, j, k)) - ph(i, j, k - 2)) / h2;
    else
        o[2] = (ph(i, j, k - 1) - ph(i, j, k + 1)) / h2;
}

// node moments: CIC sums of 1 and v per species (double atomics), into the
// slice of the sample's rf phase bin
__global__ void k_moments64(Geo g, const double4* pos, const double4* vel, const unsigned long long* nslot, int sp,
                            double* mom, double* mke, const int* bin, size_t nodes)
{
    const unsigned long long n = nslot[sp];
    mom += (size_t)*bin * 4 * nodes;
    mke += (size_t)*bin * nodes;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const double4 P = pos[q];
        if (P.w < 0.0) continue;
        const double4 V = vel[q];
        const double v2 = (V.x * V.x + V.y * V.y) + V.z * V.z;
        const double x[3] = {P.x, P.y, P.z};
        int c[3];
        double f[3];
        long long w[3][2];
        locate(g, x, c, f);
        qweights(f, w);
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int di = 0; di < 2; ++di) {
                    const double wt = (double)(w[0][di] * w[1][dy] * w[2][dz]) * 0x1p-42;
                    if (wt == 0.0) continue;
                    const size_t node = node_at(g, c[0] + di, c[1] + dy, c[2] + dz);
                    double* m = mom + 4 * node;
                    atomicAdd(m, wt);
                    atomicAdd(m + 1, wt * V.x);
                    atomicAdd(m + 2, wt * V.y);
                    atomicAdd(m + 3, wt * V.z);
                    atomicAdd(mke + node, wt * v2);
                }
    }
}

Geo geo(const pic_ctx* c) { return Geo{c->nx, c->ny, c->nz, c->dx, c->Lx, c->Ly, c->Lz}; }


// Initial plasma drawn from the run's seed, the same definition the oracle
// states: particle id p takes three uniforms at a time from its stream (p,
// step 0, kPurInitPos) for a point u L until it lies farther than 1.5 radii
// from every grain (minimum image in x and y; at most 64 tries, else the last
// point), and three normals from (p, 0, kPurInitVel) times sqrt(T e / m).
// Only the grains listed for the point's cell are tested: a point within
// 1.5 r < dx of a grain lies in the grain's 3x3x3 region, whose cells list it.
// The FP64 result is converted to the mixed layout exactly as the host upload
// converts host arrays.
struct InitP {
    Geo g;
    uint2 key;
    int64_t n;
    uint32_t id0;
    double vth, vs;              // thermal speed (m/s); dt/dx (mixed velocities in cells/step)
    const int* cell_ng;
    const int* cell_g;
    const double* gpos;
    const double* grad;
    double4* pos64;
    double4* vel64;
    float4* pos32;
    float4* vel32;
};

__device__ bool near_grain(const InitP& p, const double x[3])
{
    int c[3];
    double f[3];
    locate(p.g, x, c, f);
    const int cell = cell_of(p.g, c);
    const int ng = p.cell_ng[cell];
    const double L[3] = {p.g.Lx, p.g.Ly, p.g.Lz};
    for (int t = 0; t < ng; ++t) {
        const int gi = p.cell_g[cell * kMaxG + t];
        double d[3];
        for (int a = 0; a < 3; ++a) {
            d[a] = x[a] - p.gpos[3 * gi + a];
            if (a < 2 && d[a] > 0.5 * L[a]) d[a] = d[a] - L[a];
            else if (a < 2 && d[a] < -0.5 * L[a]) d[a] = d[a] + L[a];
        }
        const double rx = 1.5 * p.grad[gi];
        if (((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]) <= rx * rx) return true;
    }
    return false;
}

__global__ void k_init_plasma(const InitP p)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < p.n; q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t id = p.id0 + (uint32_t)q;
        const double L[3] = {p.g.Lx, p.g.Ly, p.g.Lz};
        double x[3];
        RStream rp(id, 0u, kPurInitPos, p.key);
        for (int t = 0; t < 64; ++t) {
            for (int a = 0; a < 3; ++a) x[a] = u01d(rp.next()) * L[a];
            if (!near_grain(p, x)) break;
        }
        double nv[3], v[3];
        RStream rv(id, 0u, kPurInitVel, p.key);
        gauss3(rv, nv);
        for (int a = 0; a < 3; ++a) v[a] = p.vth * nv[a];
        int c[3];
        double f[3];
        locate(p.g, x, c, f);
        if (p.pos64) {
            p.pos64[q] = make_double4(x[0], x[1], x[2], (double)cell_of(p.g, c));
            p.vel64[q] = make_double4(v[0], v[1], v[2], (double)id);
        } else {
            float o[3];
            for (int a = 0; a < 3; ++a) o[a] = fminf((float)f[a], 0.99999994f);
            const int cell = c[0] | (c[1] << 10) | (c[2] << 20);
            p.pos32[q] = make_float4(o[0], o[1], o[2], __int_as_float(cell));
            p.vel32[q] = make_float4((float)(v[0] * p.vs), (float)(v[1] * p.vs), (float)(v[2] * p.vs),
                                     __uint_as_float(id));
        }
    }
}

// Caller-supplied particles (x, v in SI as 3 doubles each, uint32 ids) into the
// run's records, particle q of the arrays to slot q0 + q: the same conversion
// as k_init_plasma's (cell and in-cell offset by `locate`; mixed velocities in
// cells per step), checked as pic_init requires (finite, 0 <= x < Lx,
// 0 <= y < Ly, 0 <= z <= Lz); a bad particle sets *bad.  *max_id takes the
// largest id.  The arrays may be host memory the device reads directly.
struct StageP {
    Geo g;
    double vs;
    const double* x;
    const double* v;
    const uint32_t* id;
    int64_t n, q0;
    double4* pos64;
    double4* vel64;
    float4* pos32;
    float4* vel32;
    unsigned int* bad;
    unsigned int* max_id;
};

__global__ void k_stage_particles(const StageP p)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < p.n; q += (int64_t)gridDim.x * blockDim.x) {
        const double x[3] = {p.x[3 * q], p.x[3 * q + 1], p.x[3 * q + 2]};
        const double v[3] = {p.v[3 * q], p.v[3 * q + 1], p.v[3 * q + 2]};
        const uint32_t id = p.id[q];
        atomicMax(p.max_id, id);
        bool ok = true;
        for (int a = 0; a < 3; ++a) ok = ok && isfinite(x[a]) && isfinite(v[a]);
        ok = ok && x[0] >= 0.0 && x[0] < p.g.Lx && x[1] >= 0.0 && x[1] < p.g.Ly && x[2] >= 0.0 && x[2] <= p.g.Lz;
        if (!ok) {
            atomicOr(p.bad, 1u);
            continue;
        }
        int c[3];
        double f[3];
        locate(p.g, x, c, f);
        const int64_t d = p.q0 + q;
        if (p.pos64) {
            p.pos64[d] = make_double4(x[0], x[1], x[2], (double)cell_of(p.g, c));
            p.vel64[d] = make_double4(v[0], v[1], v[2], (double)id);
        } else {
            float o[3];
            for (int a = 0; a < 3; ++a) o[a] = fminf((float)f[a], 0.99999994f);
            const int cell = c[0] | (c[1] << 10) | (c[2] << 20);
            p.pos32[d] = make_float4(o[0], o[1], o[2], __int_as_float(cell));
            p.vel32[d] = make_float4((float)(v[0] * p.vs), (float)(v[1] * p.vs), (float)(v[2] * p.vs),
                                     __uint_as_float(id));
        }
    }
}
}  // namespace

void launch_stage_particles(pic_ctx* c, int sp, const double* x, const double* v, const uint32_t* id, int64_t n,
                            int64_t q0, unsigned int* bad, unsigned int* max_id)
{
    if (n <= 0) return;
    StageP p;
    p.g = Geo{c->nx, c->ny, c->nz, c->dx, c->Lx, c->Ly, c->Lz};
    p.vs = c->dt / c->dx;
    p.x = x;
    p.v = v;
    p.id = id;
    p.n = n;
    p.q0 = q0;
    const bool mixed = c->prec == PIC_MIXED;
    p.pos64 = mixed ? nullptr : (double4*)c->pos[sp];
    p.vel64 = mixed ? nullptr : (double4*)c->vel[sp];
    p.pos32 = mixed ? (float4*)c->pos[sp] : nullptr;
    p.vel32 = mixed ? (float4*)c->vel[sp] : nullptr;
    p.bad = bad;
    p.max_id = max_id;
    k_stage_particles<<<grid_for(n, 256, 152 * 16), 256, 0, c->stream>>>(p);
    c->launches += 1;
}

void launch_push64(pic_ctx* c)
{
    for (int sp = 0; sp < 2; ++sp) {
        P64 p;
        p.nx = c->nx; p.ny = c->ny; p.nz = c->nz;
        p.dx = c->dx; p.Lx = c->Lx; p.Ly = c->Ly; p.Lz = c->Lz;
        p.M = c->md_sub > 0 ? c->md_sub : 1;
        p.dt = c->dt;
        p.dtm = c->dt / (double)p.M;
        p.sp = sp;
        p.qmdt = c->qm[sp] * c->dt;
        p.qmdtm = c->qm[sp] * p.dtm;
        p.hm = c->hm[sp];
        p.pnull = c->pnull[sp];
        p.nu_max = c->nu_max[sp];
        p.de = c->de[sp];
        p.n_gas = c->n_gas;
        p.sig_n = c->sig_n;
        p.eps_exc = c->eps_exc;
        p.eps_ion = c->eps_ion;
        p.mr2 = (2.0 * kME) / kMAR;
        p.kc = 1.0 / (4.0 * kPI * kEPS0);
        p.n_xs = c->n_xs;
        p.xs = c->xs64;
        p.key = c->key;
        p.step = c->d_step;
        p.flags = c->flags;
        p.ng = c->ng;
        p.gpos = c->gpos; p.grad = c->grad; p.gcell = c->gcell; p.gq = c->gq; p.gtab = c->gtab; p.gabs = c->gabs;
        p.cell_ng = c->cell_ng; p.cell_g = c->cell_g;
        p.ex = c->e64; p.ey = c->e64 + c->nodes; p.ez = c->e64 + 2 * c->nodes;
        p.rq = c->rq;
        p.pos = (double4*)c->pos[sp];
        p.vel = (double4*)c->vel[sp];
        p.nslot = c->d_nslot;
        p.cnt = c->d_cnt;
        p.err = c->d_err;
        p.child = c->d_child;
        p.child_cap = (unsigned long long)c->child_cap;
        p.nch = c->d_nch;
        k_push64<<<grid_for(c->cap[sp], 128, 152 * 16), 128, 0, c->stream>>>(p);
        c->launches += 1;
    }
}

void launch_children64(pic_ctx* c)
{
    k_children64<<<64, 256, 0, c->stream>>>(geo(c), c->d_child, c->d_nch, (unsigned long long)c->child_cap,
                                              c->d_nslot, c->d_next_id,
                                              (double4*)c->pos[0], (double4*)c->vel[0], (double4*)c->pos[1],
                                              (double4*)c->vel[1], c->cap[0], c->cap[1], c->rq, c->d_err);
    k_children_finish<<<1, 1, 0, c->stream>>>(c->d_nch, (unsigned long long)c->child_cap, c->d_nslot, c->d_next_id,
                                              c->cap[0], c->cap[1], c->d_step);
    c->launches += 2;
}

void launch_deposit64(pic_ctx* c)
{
    for (int sp = 0; sp < 2; ++sp)
        k_deposit64<<<grid_for(c->cap[sp], 256, 152 * 8), 256, 0, c->stream>>>(geo(c), (const double4*)c->pos[sp],
                                                                               c->d_nslot, sp, c->rq);
    c->launches += 2;
}

void launch_efield64(pic_ctx* c)
{
    k_efield64<<<grid_for((int64_t)c->nodes, 256, 152 * 8), 256, 0, c->stream>>>(c->nx, c->ny, c->nz, c->dx, c->phi,
                                                                                c->e64, c->e64 + c->nodes,
                                                                                c->e64 + 2 * c->nodes);
    c->launches += 1;
}

void launch_moments64(pic_ctx* c)
{
    for (int sp = 0; sp < 2; ++sp)
        k_moments64<<<grid_for(c->cap[sp], 256, 152 * 8), 256, 0, c->stream>>>(
            geo(c), (const double4*)c->pos[sp], (const double4*)c->vel[sp], c->d_nslot, sp, c->mom[sp], c->mke[sp],
            c->d_bin, c->nodes);
    c->launches += 2;
}

void launch_grains(pic_ctx* c)
{
    if (c->ng == 0) return;
    k_grains<<<(c->ng + 63) / 64, 64, 0, c->stream>>>(geo(c), c->ng, kQE * c->W, c->gabs, c->gpos, c->gq, c->gq32,
                                                     c->rq);
    c->launches += 1;
}

void launch_grain_table(pic_ctx* c, int gi)
{
    k_grain_table<<<1, 64, 0, c->stream>>>(c->nx, c->ny, c->nz, c->dx, c->phi, c->gcell, gi, c->gtab);
    c->launches += 1;
}
void launch_green_block(pic_ctx* c, int k, double* blk)
{
    k_green_block<<<1, 352, 0, c->stream>>>(c->nx, c->ny, c->nz, c->phi, k, blk);
    c->launches += 1;
}

void launch_grain_tables_sup(pic_ctx* c, const double* blk, const int* plane)
{
    if (c->ng == 0) return;
    k_grain_table_sup<<<c->ng, 64, 0, c->stream>>>(geo(c), c->gpos, c->gcell, blk, plane, c->gtab);
    c->launches += 1;
}

void launch_init_plasma(pic_ctx* c, int sp, int64_t n, uint32_t id0, double t_ev)
{
    if (n <= 0) return;
    InitP p;
    p.g = Geo{c->nx, c->ny, c->nz, c->dx, c->Lx, c->Ly, c->Lz};
    p.key = c->key;
    p.n = n;
    p.id0 = id0;
    p.vth = sqrt((t_ev * kQE) / (sp == 0 ? kME : kMAR));
    p.vs = c->dt / c->dx;
    p.cell_ng = c->cell_ng;
    p.cell_g = c->cell_g;
    p.gpos = c->gpos;
    p.grad = c->grad;
    const bool mixed = c->prec == PIC_MIXED;
    p.pos64 = mixed ? nullptr : (double4*)c->pos[sp];
    p.vel64 = mixed ? nullptr : (double4*)c->vel[sp];
    p.pos32 = mixed ? (float4*)c->pos[sp] : nullptr;
    p.vel32 = mixed ? (float4*)c->vel[sp] : nullptr;
    k_init_plasma<<<grid_for(n, 256, 152 * 16), 256, 0, c->stream>>>(p);
    c->launches += 1;
}

}  // namespace pic

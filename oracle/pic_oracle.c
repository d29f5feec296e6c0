/*
 * Oracle for the PIC-MCC/PPPM particle cycle (arXiv:1801.00972, Sec. III).
 *
 * TEST INFRASTRUCTURE ONLY: a plain FP64 CPU restatement of the method that
 * the CUDA library is checked against.  Only tests, the smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code with the library.
 * Build with -ffp-contract=off so that every product and sum rounds on its
 * own (no fused multiply-add), which keeps the arithmetic order written here
 * the arithmetic that runs.
 *
 * One time step, from positions x_k and velocities v_{k-1/2} (Eqs. 1-2):
 *   1. E at the mesh nodes from Phi_k by central differences (Eq. 4; Sec. III
 *      "electric field ... by finite differences").
 *   2. every particle: CIC gather of E (Sec. III, same weighting as the
 *      deposit); velocity kick (Eq. 2) and drift (Eq. 1).  A particle whose
 *      cell is in an MD region (grain cell + direct neighbours) instead takes
 *      md_sub substeps of dt/md_sub with E = E_PIC - E_PIC^dust + E_MD^dust
 *      (Eqs. 5-6) and an absorption test against the grains after each
 *      substep.  Electrodes absorb; x and y are periodic.
 *   3. null-collision Monte Carlo collisions with the argon background
 *      (Table I: e elastic, excitation, ionization; Ar+ elastic, charge
 *      exchange); ionization appends an electron and an ion.
 *   4. grain charges Q = e W (N_ion,abs - N_e,abs) (integer charge steps).
 *   5. CIC deposit of all particles and of the grain charges into rho (Sec.
 *      III, box shape, cell-corner nodes), in exact integer fixed point.
 *   6. exact solve of the discrete Poisson equation (Eq. 3), periodic in x
 *      and y, Dirichlet electrodes in z (the paper's LU back-solve gives the
 *      same discrete solution; here a DFT in x,y and a tridiagonal solve in
 *      z do it).
 */
#include "pic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

#define QE    1.602176634e-19      /* elementary charge, C          */
#define EPS0  8.8541878128e-12     /* vacuum permittivity, F/m      */
#define ME    9.1093837015e-31     /* electron mass, kg             */
#define AMU   1.66053906660e-27    /* atomic mass unit, kg          */
#define KB    1.380649e-23         /* Boltzmann constant, J/K       */
#define MAR   (39.948 * AMU)       /* argon mass, kg                */
#define PI_D  3.14159265358979323846
#define WQ    16384                /* fixed-point CIC weight units per axis (2^14) */
#define MAXG  8                    /* grains per MD cell */

enum { PUR_MCC = 1, PUR_DIR = 2, PUR_NEUTRAL = 3, PUR_CHILD_DIR = 4, PUR_CHILD_NEUTRAL = 5,
       PUR_COUL_ORDER = 6, PUR_COUL_EE = 7, PUR_COUL_II = 8, PUR_COUL_EI = 9,
       PUR_INIT_POS = 10, PUR_INIT_VEL = 11 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11) */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform on (0,1): (u + 1/2) 2^-32, exact in double */
static double u01(uint32_t u) { return ((double)u + 0.5) * 2.3283064365386962890625e-10; }

/* Natural logarithm from +,-,*,/ only: x = m 2^e with m in [sqrt(1/2), sqrt(2)),
 * ln m = 2 atanh(s), s = (m-1)/(m+1), by its odd power series up to s^23. */
double orc_ln(double x)
{
    int e;
    double m = frexp(x, &e);
    if (m < 0.70710678118654752440) { m = m * 2.0; e = e - 1; }
    double s = (m - 1.0) / (m + 1.0);
    double s2 = s * s;
    double p = 1.0 / 23.0;
    p = p * s2 + 1.0 / 21.0;
    p = p * s2 + 1.0 / 19.0;
    p = p * s2 + 1.0 / 17.0;
    p = p * s2 + 1.0 / 15.0;
    p = p * s2 + 1.0 / 13.0;
    p = p * s2 + 1.0 / 11.0;
    p = p * s2 + 1.0 / 9.0;
    p = p * s2 + 1.0 / 7.0;
    p = p * s2 + 1.0 / 5.0;
    p = p * s2 + 1.0 / 3.0;
    p = p * s2 + 1.0;
    double t1 = (double)e * 0.69314718055994530942;
    double t2 = (2.0 * s) * p;
    return t1 + t2;
}

/* A stream of uniforms for one (particle, step, purpose): Philox calls with
 * the fourth counter word counting the calls. */
typedef struct { uint32_t ctr[4]; uint32_t key[2]; uint32_t buf[4]; int pos; } rstream;

static void rs_init(rstream* r, uint32_t id, uint32_t step, uint32_t purpose, const uint32_t key[2])
{
    r->ctr[0] = id; r->ctr[1] = step; r->ctr[2] = purpose; r->ctr[3] = 0;
    r->key[0] = key[0]; r->key[1] = key[1]; r->pos = 4;
}
static uint32_t rs_next(rstream* r)
{
    if (r->pos == 4) { orc_philox4x32_10(r->ctr, r->key, r->buf); r->ctr[3] += 1; r->pos = 0; }
    return r->buf[r->pos++];
}
/* a point uniform in the square (-1,1)^2 */
static void rs_pair(rstream* r, double* a, double* b)
{
    uint32_t ua = rs_next(r), ub = rs_next(r);
    *a = 2.0 * u01(ua) - 1.0;
    *b = 2.0 * u01(ub) - 1.0;
}
/* isotropic unit vector, Marsaglia (1972) disk rejection */
static void rs_iso(rstream* r, double out[3])
{
    for (int t = 0; t < 128; ++t) {
        double a, b;
        rs_pair(r, &a, &b);
        double s = a * a + b * b;
        if (s < 1.0) {
            double q = 2.0 * sqrt(1.0 - s);
            out[0] = a * q; out[1] = b * q; out[2] = 1.0 - 2.0 * s;
            return;
        }
    }
    out[0] = 0.0; out[1] = 0.0; out[2] = 1.0;
}
/* two standard normals, Marsaglia polar method */
static void rs_gauss2(rstream* r, double* n1, double* n2)
{
    for (int t = 0; t < 128; ++t) {
        double a, b;
        rs_pair(r, &a, &b);
        double s = a * a + b * b;
        if (s < 1.0) {
            double f = sqrt((-2.0 * orc_ln(s)) / s);
            *n1 = a * f; *n2 = b * f;
            return;
        }
    }
    *n1 = 0.0; *n2 = 0.0;
}
static void rs_gauss3(rstream* r, double out[3])
{
    double d;
    rs_gauss2(r, &out[0], &out[1]);
    rs_gauss2(r, &out[2], &d);
}

void orc_iso_dir(uint32_t id, uint32_t step, uint32_t purpose, const uint32_t key[2], double out[3])
{
    rstream r; rs_init(&r, id, step, purpose, key); rs_iso(&r, out);
}
void orc_gauss3(uint32_t id, uint32_t step, uint32_t purpose, const uint32_t key[2], double out[3])
{
    rstream r; rs_init(&r, id, step, purpose, key); rs_gauss3(&r, out);
}

/* ------------------------------------------------------------------------ */
/* Exact discrete Poisson solve (Eq. 3) on the node mesh                     */
/* ------------------------------------------------------------------------ */
/* 2-D DFT of one plane (nx fastest), sign -1 forward, +1 backward (no 1/n):
 * X(m, m2) = sum_{i,j} x(i, j) exp(sign 2 pi i (m i / nx + m2 j / ny)).
 * Plain O(n^2) sums for any size; planes whose sides are both powers of two
 * use the radix-2 fast transform below, which computes the same sums. */
static void dft2(int nx, int ny, const double* cx, const double* sx, const double* cy,
                 const double* sy, double sign, const double* ire, const double* iim,
                 double* ore, double* oim, double* tre, double* tim)
{
    for (int j = 0; j < ny; ++j)
        for (int m = 0; m < nx; ++m) {
            double ar = 0.0, ai = 0.0;
            for (int i = 0; i < nx; ++i) {
                int t = (int)(((long)m * i) % nx);
                double c = cx[t], s = sign * sx[t];
                double xr = ire[j * nx + i], xi = iim ? iim[j * nx + i] : 0.0;
                ar += xr * c - xi * s;
                ai += xr * s + xi * c;
            }
            tre[j * nx + m] = ar; tim[j * nx + m] = ai;
        }
    for (int m2 = 0; m2 < ny; ++m2)
        for (int m = 0; m < nx; ++m) {
            double ar = 0.0, ai = 0.0;
            for (int j = 0; j < ny; ++j) {
                int t = (int)(((long)m2 * j) % ny);
                double c = cy[t], s = sign * sy[t];
                double xr = tre[j * nx + m], xi = tim[j * nx + m];
                ar += xr * c - xi * s;
                ai += xr * s + xi * c;
            }
            ore[m2 * nx + m] = ar; oim[m2 * nx + m] = ai;
        }
}

static int pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* Radix-2 Cooley-Tukey fast Fourier transform of n = 2^q complex values at
 * stride `st`, in place: the bit-reversal permutation, then q passes of
 * butterflies (a, b) -> (a + w b, a - w b) over blocks of length 2, 4, ..., n
 * with w = exp(sign 2 pi i t / len); c[t], s[t] = cos, sin(2 pi t / n). */
static void fft1(int n, double* re, double* im, size_t st, double sign, const double* c, const double* s)
{
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i * st]; re[i * st] = re[j * st]; re[j * st] = t;
            t = im[i * st]; im[i * st] = im[j * st]; im[j * st] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len >> 1, step = n / len;
        for (int b = 0; b < n; b += len)
            for (int k = 0; k < half; ++k) {
                const double wr = c[k * step], wi = sign * s[k * step];
                const size_t ia = (size_t)(b + k) * st, ib = (size_t)(b + k + half) * st;
                const double xr = re[ib] * wr - im[ib] * wi;
                const double xi = re[ib] * wi + im[ib] * wr;
                re[ib] = re[ia] - xr; im[ib] = im[ia] - xi;
                re[ia] = re[ia] + xr; im[ia] = im[ia] + xi;
            }
    }
}

/* the 2-D transform of one plane in place: rows (x), then columns (y) */
static void plane_transform(int nx, int ny, const double* cx, const double* sx, const double* cy,
                            const double* sy, double sign, double* re, double* im, double* tre, double* tim)
{
    if (pow2(nx) && pow2(ny)) {
        for (int j = 0; j < ny; ++j) fft1(nx, re + (size_t)j * nx, im + (size_t)j * nx, 1, sign, cx, sx);
        for (int i = 0; i < nx; ++i) fft1(ny, re + i, im + i, (size_t)nx, sign, cy, sy);
        return;
    }
    dft2(nx, ny, cx, sx, cy, sy, sign, re, im, tre, tim, tre + (size_t)nx * ny, tim + (size_t)nx * ny);
    memcpy(re, tre, sizeof(double) * (size_t)nx * ny);
    memcpy(im, tim, sizeof(double) * (size_t)nx * ny);
}

/* Tridiagonal solve of one Fourier mode (Thomas): u_{k-1} + d u_k + u_{k+1} = r_k
 * for k = 1..n with u_0 = u_{n+1} = 0 (electrode terms already moved into r);
 * cp, rr, ri are scratch of n + 1 values. */
static void thomas_mode(int n, double d, double* rr, double* ri, double* cp)
{
    cp[1] = 1.0 / d;
    rr[1] = rr[1] / d; ri[1] = ri[1] / d;
    for (int k = 2; k <= n; ++k) {
        double mm = d - cp[k - 1];
        cp[k] = 1.0 / mm;
        rr[k] = (rr[k] - rr[k - 1]) / mm;
        ri[k] = (ri[k] - ri[k - 1]) / mm;
    }
    for (int k = n - 1; k >= 1; --k) {
        rr[k] = rr[k] - cp[k] * rr[k + 1];
        ri[k] = ri[k] - cp[k] * ri[k + 1];
    }
}

/* Solve (sum of the six neighbours - 6 phi)/dx^2 = -f on the interior nodes
 * k = 1..nz-1, periodic in x,y, phi(k=0) = v_bot, phi(k=nz) = v_top.
 * f and phi are node arrays indexed (k*ny + j)*nx + i.  The discrete Fourier
 * transform in x and y diagonalises the periodic part, leaving one
 * tridiagonal system in z per mode.  Planes and modes are independent, so
 * they are shared among OpenMP threads; the result does not depend on the
 * thread count. */
int orc_poisson(int nx, int ny, int nz, double dx, const double* f, double v_bot,
                double v_top, double* phi)
{
    const int P = nx * ny;
    const size_t N = (size_t)P * (size_t)(nz + 1);
    double* re = (double*)calloc(N, sizeof(double));
    double* im = (double*)calloc(N, sizeof(double));
    double* cx = (double*)malloc(sizeof(double) * nx);
    double* sx = (double*)malloc(sizeof(double) * nx);
    double* cy = (double*)malloc(sizeof(double) * ny);
    double* sy = (double*)malloc(sizeof(double) * ny);
    if (!re || !im || !cx || !sx || !cy || !sy) return -1;
    for (int t = 0; t < nx; ++t) { cx[t] = cos(2.0 * PI_D * t / nx); sx[t] = sin(2.0 * PI_D * t / nx); }
    for (int t = 0; t < ny; ++t) { cy[t] = cos(2.0 * PI_D * t / ny); sy[t] = sin(2.0 * PI_D * t / ny); }
    int bad = 0;

    /* right-hand side -dx^2 f, transformed plane by plane */
    #pragma omp parallel reduction(|:bad)
    {
        double* t2 = (double*)malloc(sizeof(double) * 4 * (size_t)P);
        if (!t2) bad = 1;
        #pragma omp for schedule(static)
        for (int k = 1; k < nz; ++k) {
            if (!t2) continue;
            double* pr = re + (size_t)k * P;
            for (int p = 0; p < P; ++p) pr[p] = -(dx * dx) * f[(size_t)k * P + p];
            plane_transform(nx, ny, cx, sx, cy, sy, -1.0, pr, im + (size_t)k * P, t2, t2 + 2 * (size_t)P);
        }
        free(t2);
    }

    /* one tridiagonal system per Fourier mode:
     * u_{k-1} + d u_k + u_{k+1} = r_k,  d = 2 cos(th1) + 2 cos(th2) - 6 */
    #pragma omp parallel reduction(|:bad)
    {
        double* cp = (double*)malloc(sizeof(double) * (nz + 1));
        double* rr = (double*)malloc(sizeof(double) * (nz + 1));
        double* ri = (double*)malloc(sizeof(double) * (nz + 1));
        if (!cp || !rr || !ri) bad = 1;
        #pragma omp for schedule(static)
        for (int p = 0; p < P; ++p) {
            if (!cp || !rr || !ri) continue;
            const int m1 = p % nx, m2 = p / nx;
            const double d = (2.0 * cx[m1] + 2.0 * cy[m2]) - 6.0;
            const double b0 = (p == 0) ? (double)P * v_bot : 0.0;
            const double bn = (p == 0) ? (double)P * v_top : 0.0;
            const int n = nz - 1;
            for (int k = 1; k <= n; ++k) { rr[k] = re[(size_t)k * P + p]; ri[k] = im[(size_t)k * P + p]; }
            rr[1] -= b0;
            rr[n] -= bn;
            thomas_mode(n, d, rr, ri, cp);
            for (int k = 1; k <= n; ++k) { re[(size_t)k * P + p] = rr[k]; im[(size_t)k * P + p] = ri[k]; }
        }
        free(cp); free(rr); free(ri);
    }

    /* back to space */
    #pragma omp parallel reduction(|:bad)
    {
        double* t2 = (double*)malloc(sizeof(double) * 4 * (size_t)P);
        if (!t2) bad = 1;
        #pragma omp for schedule(static)
        for (int k = 1; k < nz; ++k) {
            if (!t2) continue;
            double* pr = re + (size_t)k * P;
            plane_transform(nx, ny, cx, sx, cy, sy, +1.0, pr, im + (size_t)k * P, t2, t2 + 2 * (size_t)P);
            for (int q = 0; q < P; ++q) phi[(size_t)k * P + q] = pr[q] / (double)P;
        }
        free(t2);
    }
    for (int q = 0; q < P; ++q) { phi[q] = v_bot; phi[(size_t)nz * P + q] = v_top; }
    free(re); free(im); free(cx); free(sx); free(cy); free(sy);
    return bad ? -1 : 0;
}

/* E = -grad phi at the nodes (Eq. 4): central differences, periodic in x,y;
 * second-order one-sided differences on the electrode planes. */
void orc_efield(int nx, int ny, int nz, double dx, const double* phi, double* ex, double* ey, double* ez)
{
    const double h2 = 2.0 * dx;
    #pragma omp parallel for schedule(static)
    for (int k = 0; k <= nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t n = ((size_t)k * ny + j) * nx + i;
                int ip = (i + 1) % nx, im = (i + nx - 1) % nx;
                int jp = (j + 1) % ny, jm = (j + ny - 1) % ny;
                ex[n] = (phi[((size_t)k * ny + j) * nx + im] - phi[((size_t)k * ny + j) * nx + ip]) / h2;
                ey[n] = (phi[((size_t)k * ny + jm) * nx + i] - phi[((size_t)k * ny + jp) * nx + i]) / h2;
                const size_t P = (size_t)nx * ny;
                if (k == 0)
                    ez[n] = ((3.0 * phi[n] - 4.0 * phi[n + P]) + phi[n + 2 * P]) / h2;
                else if (k == nz)
                    ez[n] = ((4.0 * phi[n - P] - 3.0 * phi[n]) - phi[n - 2 * P]) / h2;
                else
                    ez[n] = (phi[n - P] - phi[n + P]) / h2;
            }
}

/* ------------------------------------------------------------------------ */
/* simulation state                                                          */
/* ------------------------------------------------------------------------ */
typedef struct { uint32_t parent; double x[3], ve[3], vi[3]; } child_rec;

struct orc_sim {
    orc_cfg c;
    double Lx, Ly, Lz;
    double qm[2], hm[2];           /* q/m and (m/2)/e per species */
    double pnull[2];
    uint32_t key[2];
    int64_t n[2], cap[2];
    double* x[2];
    double* v[2];
    uint32_t* id[2];
    int64_t* rq;                   /* fixed-point charge per node */
    double *phi, *ex, *ey, *ez;
    double* xs;                    /* owned copy of the tables */
    double *gpos, *grad, *gq, *gtab;
    int64_t* gabs;                 /* [g][species] */
    int* cell_ng;
    int* cell_g;
    int64_t step;
    uint32_t next_id;
    int64_t cnt[ORC_C_N];
    child_rec* ch; int64_t nch, capch;
    double* mom[2];                /* [phase bin][node][4]: count, count*vx, count*vy, count*vz */
    double* mphi;                  /* [phase bin][node] */
    double* mke[2];                /* [phase bin][node]: count * |v|^2 */
    int64_t msteps;
    int64_t* bsteps;               /* samples per phase bin */
    int nph;                       /* phase bins (1 without phase resolution) */
    double* fine[2];               /* [fine cell][4]: count, sum vx, sum vy, sum vz */
    size_t nfine;
    int64_t* eepf;                 /* [k][bin] electron counts */
    int64_t eepf_steps;
};

static size_t nodes_of(const orc_sim* s) { return (size_t)s->c.nx * s->c.ny * (s->c.nz + 1); }
static size_t cells_of(const orc_sim* s) { return (size_t)s->c.nx * s->c.ny * s->c.nz; }

/* cell indices and in-cell fractions of a position */
static void locate(const orc_sim* s, const double* p, int c[3], double f[3])
{
    const int nn[3] = { s->c.nx, s->c.ny, s->c.nz };
    for (int a = 0; a < 3; ++a) {
        double q = p[a] / s->c.dx;
        int i = (int)floor(q);
        if (i > nn[a] - 1) i = nn[a] - 1;
        if (i < 0) i = 0;
        c[a] = i;
        f[a] = q - (double)i;
    }
}
/* per-axis fixed-point CIC weights (lower corner, upper corner), summing to 2^14 */
static void qweights(const double f[3], int64_t w[3][2])
{
    for (int a = 0; a < 3; ++a) {
        int64_t q = (int64_t)rint(f[a] * (double)WQ);
        if (q < 0) q = 0;
        if (q > WQ) q = WQ;
        w[a][0] = WQ - q; w[a][1] = q;
    }
}
static size_t node_at(const orc_sim* s, int i, int j, int k)
{
    i %= s->c.nx; j %= s->c.ny;
    return ((size_t)k * s->c.ny + j) * s->c.nx + i;
}
static size_t cell_index(const orc_sim* s, const int c[3])
{
    return ((size_t)c[2] * s->c.ny + c[1]) * s->c.nx + c[0];
}

static void deposit_one(const orc_sim* s, int64_t* rq, const double* p, int64_t charge)
{
    int c[3]; double f[3]; int64_t w[3][2];
    locate(s, p, c, f);
    qweights(f, w);
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dxi = 0; dxi < 2; ++dxi)
            {
                const int64_t add = charge * (w[0][dxi] * w[1][dy] * w[2][dz]);
                int64_t* r = rq + node_at(s, c[0] + dxi, c[1] + dy, c[2] + dz);
                #pragma omp atomic
                *r += add;
            }
}

/* CIC gather of a node vector field with the same fixed-point weights */
static void gather(const orc_sim* s, const double* fx, const double* fy, const double* fz,
                   const int c[3], const int64_t w[3][2], double E[3])
{
    E[0] = 0.0; E[1] = 0.0; E[2] = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dxi = 0; dxi < 2; ++dxi) {
                double wt = (double)(w[0][dxi] * w[1][dy] * w[2][dz]) * 0x1p-42;
                size_t n = node_at(s, c[0] + dxi, c[1] + dy, c[2] + dz);
                E[0] = E[0] + wt * fx[n];
                E[1] = E[1] + wt * fy[n];
                E[2] = E[2] + wt * fz[n];
            }
}

/* minimum-image separation from grain g */
static void grain_sep(const orc_sim* s, int g, const double* p, double d[3])
{
    const double L[2] = { s->Lx, s->Ly };
    for (int a = 0; a < 2; ++a) {
        double q = p[a] - s->gpos[3 * g + a];
        if (q > 0.5 * L[a]) q = q - L[a];
        else if (q < -0.5 * L[a]) q = q + L[a];
        d[a] = q;
    }
    d[2] = p[2] - s->gpos[3 * g + 2];
}

/* Eqs. 5-6 inside an MD region: subtract each near grain's mesh field (its
 * unit-charge node field table times Q, CIC-gathered) and add its Coulomb
 * field Q (x - x_g) / (4 pi eps0 |x - x_g|^3). */
static void md_correct(const orc_sim* s, const double* p, const int c[3], const int64_t w[3][2], double E[3])
{
    const size_t cell = cell_index(s, c);
    const double kc = 1.0 / (4.0 * PI_D * EPS0);
    for (int t = 0; t < s->cell_ng[cell]; ++t) {
        const int g = s->cell_g[cell * MAXG + t];
        const int gc[3] = { (int)floor(s->gpos[3 * g] / s->c.dx), (int)floor(s->gpos[3 * g + 1] / s->c.dx),
                            (int)floor(s->gpos[3 * g + 2] / s->c.dx) };
        double Ed[3] = { 0.0, 0.0, 0.0 };
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dxi = 0; dxi < 2; ++dxi) {
                    double wt = (double)(w[0][dxi] * w[1][dy] * w[2][dz]) * 0x1p-42;
                    int li = ((c[0] + dxi - gc[0] + 1) % s->c.nx + s->c.nx) % s->c.nx;
                    int lj = ((c[1] + dy - gc[1] + 1) % s->c.ny + s->c.ny) % s->c.ny;
                    int lk = c[2] + dz - gc[2] + 1;
                    const double* tv = s->gtab + ((size_t)g * 64 + (lk * 4 + lj) * 4 + li) * 3;
                    Ed[0] = Ed[0] + wt * tv[0];
                    Ed[1] = Ed[1] + wt * tv[1];
                    Ed[2] = Ed[2] + wt * tv[2];
                }
        double d[3];
        grain_sep(s, g, p, d);
        double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        double Q = s->gq[g];
        double coef = 0.0;
        if (r2 > 0.0) { double r = sqrt(r2); coef = (Q * kc) / (r2 * r); }
        for (int a = 0; a < 3; ++a) E[a] = (E[a] - Q * Ed[a]) + coef * d[a];
    }
}

/* 0 alive, 1 lost at z=0, 2 lost at z=Lz, 3 invalid (non-finite or moved a box length) */
static int boundary(const orc_sim* s, double* p)
{
    if (!(p[2] >= 0.0)) return (p[2] < 0.0) ? 1 : 3;
    if (p[2] > s->Lz) return 2;
    const double L[2] = { s->Lx, s->Ly };
    for (int a = 0; a < 2; ++a) {
        if (p[a] < 0.0) p[a] = p[a] + L[a];
        else if (p[a] >= L[a]) p[a] = p[a] - L[a];
        if (!(p[a] >= 0.0 && p[a] <= L[a])) return 3;
    }
    return 0;
}

static int absorbed_by(const orc_sim* s, const double* p)
{
    int c[3]; double f[3];
    locate(s, p, c, f);
    const size_t cell = cell_index(s, c);
    for (int t = 0; t < s->cell_ng[cell]; ++t) {
        const int g = s->cell_g[cell * MAXG + t];
        double d[3];
        grain_sep(s, g, p, d);
        double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        if (r2 <= s->grad[g] * s->grad[g]) return g;
    }
    return -1;
}

static double xs_at(const double* tab, int n, double de, double eps)
{
    double t = eps / de;
    if (t >= (double)(n - 1)) return tab[n - 1];
    int i = (int)t;
    double fr = t - (double)i;
    return tab[i] + fr * (tab[i + 1] - tab[i]);
}

/* what one thread's particles did during a step: event counts and ionization
 * products, merged after the particle loop */
typedef struct { int64_t cnt[ORC_C_N]; child_rec* ch; int64_t nch, capch; } step_log;

static void push_child(step_log* t, const child_rec* r)
{
    if (t->nch == t->capch) {
        t->capch = t->capch ? 2 * t->capch : 64;
        t->ch = (child_rec*)realloc(t->ch, sizeof(child_rec) * t->capch);
    }
    t->ch[t->nch++] = *r;
}

static int thread_id(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

/* null-collision MCC for one particle after its push (Table I) */
static void mcc(const orc_sim* s, step_log* t, int sp, double* p, double* v, uint32_t id)
{
    const uint32_t step = (uint32_t)s->step;
    uint32_t ctr[4] = { id, step, PUR_MCC, 0 }, u[4];
    orc_philox4x32_10(ctr, s->key, u);
    if (u01(u[0]) >= s->pnull[sp]) return;
    const double ng = s->c.n_gas;
    const int nx = s->c.n_xs;
    const double sig_n = sqrt(KB * s->c.t_gas / MAR);
    if (sp == 0) {
        double v2 = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
        double eps = v2 * s->hm[0];
        double vm = sqrt(v2);
        double nu_el = (ng * xs_at(s->xs + 0 * nx, nx, s->c.de_e, eps)) * vm;
        double nu_ex = (ng * xs_at(s->xs + 1 * nx, nx, s->c.de_e, eps)) * vm;
        double nu_io = (ng * xs_at(s->xs + 2 * nx, nx, s->c.de_e, eps)) * vm;
        double R = u01(u[1]) * s->c.nu_max_e;
        double acc = nu_el;
        rstream rd; rs_init(&rd, id, step, PUR_DIR, s->key);
        double dir[3];
        if (R < acc) {
            /* elastic: isotropic, energy loss (2 m_e / M)(1 - cos chi) */
            rs_iso(&rd, dir);
            double cosx = ((dir[0] * v[0] + dir[1] * v[1]) + dir[2] * v[2]) / vm;
            double fac = 1.0 - ((2.0 * ME) / MAR) * (1.0 - cosx);
            double vn = vm * sqrt(fac);
            for (int a = 0; a < 3; ++a) v[a] = vn * dir[a];
            t->cnt[ORC_C_E_EL]++;
            return;
        }
        acc = acc + nu_ex;
        if (R < acc) {
            double e2 = eps - s->c.eps_exc;
            if (e2 < 0.0) e2 = 0.0;
            rs_iso(&rd, dir);
            double vn = sqrt(e2 / s->hm[0]);
            for (int a = 0; a < 3; ++a) v[a] = vn * dir[a];
            t->cnt[ORC_C_E_EXC]++;
            return;
        }
        acc = acc + nu_io;
        if (R < acc) {
            double e2 = eps - s->c.eps_ion;
            if (e2 < 0.0) e2 = 0.0;
            double vn = sqrt((0.5 * e2) / s->hm[0]);
            rs_iso(&rd, dir);
            child_rec cr;
            cr.parent = id;
            for (int a = 0; a < 3; ++a) { v[a] = vn * dir[a]; cr.x[a] = p[a]; }
            double d2[3], gn[3];
            rstream rc; rs_init(&rc, id, step, PUR_CHILD_DIR, s->key); rs_iso(&rc, d2);
            rstream rn; rs_init(&rn, id, step, PUR_CHILD_NEUTRAL, s->key); rs_gauss3(&rn, gn);
            for (int a = 0; a < 3; ++a) { cr.ve[a] = vn * d2[a]; cr.vi[a] = sig_n * gn[a]; }
            push_child(t, &cr);
            t->cnt[ORC_C_E_ION]++;
        }
        return;
    }
    /* ions: relative velocity to a neutral drawn from the 300 K Maxwellian */
    double gn[3];
    rstream rn; rs_init(&rn, id, step, PUR_NEUTRAL, s->key); rs_gauss3(&rn, gn);
    double vn[3] = { sig_n * gn[0], sig_n * gn[1], sig_n * gn[2] };
    double g[3] = { v[0] - vn[0], v[1] - vn[1], v[2] - vn[2] };
    double g2 = (g[0] * g[0] + g[1] * g[1]) + g[2] * g[2];
    double eps = g2 * s->hm[1];
    double gm = sqrt(g2);
    double nu_el = (ng * xs_at(s->xs + 3 * nx, nx, s->c.de_i, eps)) * gm;
    double nu_cx = (ng * xs_at(s->xs + 4 * nx, nx, s->c.de_i, eps)) * gm;
    double R = u01(u[1]) * s->c.nu_max_i;
    double acc = nu_el;
    if (R < acc) {
        /* elastic, isotropic in the centre-of-mass frame (equal masses) */
        double dir[3];
        rstream rd; rs_init(&rd, id, step, PUR_DIR, s->key); rs_iso(&rd, dir);
        for (int a = 0; a < 3; ++a) v[a] = (v[a] + vn[a]) * 0.5 + (0.5 * gm) * dir[a];
        t->cnt[ORC_C_I_EL]++;
        return;
    }
    acc = acc + nu_cx;
    if (R < acc) {
        for (int a = 0; a < 3; ++a) v[a] = vn[a];
        t->cnt[ORC_C_I_CX]++;
    }
}

static int cmp_child(const void* a, const void* b)
{
    uint32_t x = ((const child_rec*)a)->parent, y = ((const child_rec*)b)->parent;
    return (x > y) - (x < y);
}

static void grow(orc_sim* s, int sp, int64_t need)
{
    if (need <= s->cap[sp]) return;
    int64_t nc = s->cap[sp] ? s->cap[sp] : 16;
    while (nc < need) nc *= 2;
    s->x[sp] = (double*)realloc(s->x[sp], sizeof(double) * 3 * nc);
    s->v[sp] = (double*)realloc(s->v[sp], sizeof(double) * 3 * nc);
    s->id[sp] = (uint32_t*)realloc(s->id[sp], sizeof(uint32_t) * nc);
    s->cap[sp] = nc;
}

static void deposit_all(orc_sim* s)
{
    memset(s->rq, 0, sizeof(int64_t) * nodes_of(s));
    /* integer sums: any order of the additions gives the same result */
    for (int sp = 0; sp < 2; ++sp) {
        const int64_t charge = sp == 0 ? -1 : 1;
        #pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < s->n[sp]; ++q) deposit_one(s, s->rq, s->x[sp] + 3 * q, charge);
    }
    for (int g = 0; g < s->c.n_grains; ++g)
        deposit_one(s, s->rq, s->gpos + 3 * g, s->gabs[2 * g + 1] - s->gabs[2 * g + 0]);
}

static double v_bottom(const orc_sim* s)
{
    double t = (double)s->step * s->c.dt;
    return s->c.v_dc + s->c.v_rf * sin((2.0 * PI_D * s->c.f_rf) * t + s->c.phase);
}

int orc_solve(orc_sim* s)
{
    const size_t N = nodes_of(s);
    double* f = (double*)malloc(sizeof(double) * N);
    const double dx = s->c.dx;
    const double scale = (((QE * s->c.weight) / (dx * dx * dx)) * 0x1p-42) / EPS0;
    for (size_t q = 0; q < N; ++q) f[q] = (double)s->rq[q] * scale;
    int rc = orc_poisson(s->c.nx, s->c.ny, s->c.nz, dx, f, v_bottom(s), s->c.v_top, s->phi);
    free(f);
    return rc;
}

/* rf phase bin of the samples taken after the current step (t = step dt): the
 * argument 2 pi f t + phase of the electrode voltage, taken modulo 2 pi and
 * cut into nph equal bins starting at phase 0 (Sec. IV.C: electron fluxes
 * resolved in rf phase, ion fluxes averaged over the period) */
static int phase_bin(const orc_sim* s)
{
    if (s->nph == 1) return 0;
    const double t = (double)s->step * s->c.dt;
    const double u = s->c.f_rf * t + s->c.phase / (2.0 * PI_D);
    const double fr = u - floor(u);
    const int b = (int)(fr * (double)s->nph);
    return b < s->nph ? b : s->nph - 1;
}

/* Sec. IV.C: inside the MD region the paper samples densities and fluxes on
 * a grid of cubes of edge 0.08 dx instead of the PIC cells.  A particle adds
 * 1 and its velocity to the fine cell that holds it (an average over the
 * cell's volume); particles outside the box add nothing. */
static void fine_accumulate(orc_sim* s, int sp, const double* p, const double* vv)
{
    int f[3];
    for (int a = 0; a < 3; ++a) {
        const double q = (p[a] - s->c.fine_origin[a]) / s->c.fine_h;
        if (!(q >= 0.0) || !(q < (double)s->c.fine_n[a])) return;
        f[a] = (int)q;
    }
    const size_t cell = ((size_t)f[2] * (size_t)s->c.fine_n[1] + (size_t)f[1]) * (size_t)s->c.fine_n[0] + (size_t)f[0];
    double* m = s->fine[sp] + 4 * cell;
    m[0] += 1.0; m[1] += vv[0]; m[2] += vv[1]; m[3] += vv[2];
}

/* node moments (Sec. IV: time averages): CIC weights of every particle at the
 * end of a step, summed with the weight times its velocity, and phi; into the
 * phase bin of the step */
static void moments_accumulate(orc_sim* s)
{
    const size_t N = nodes_of(s);
    const int b = phase_bin(s);
    for (int sp = 0; sp < 2; ++sp)
        for (int64_t q = 0; q < s->n[sp]; ++q) {
            int c[3]; double f[3]; int64_t w[3][2];
            const double* p = s->x[sp] + 3 * q;
            const double* vv = s->v[sp] + 3 * q;
            const double v2 = (vv[0] * vv[0] + vv[1] * vv[1]) + vv[2] * vv[2];
            locate(s, p, c, f);
            qweights(f, w);
            for (int dz = 0; dz < 2; ++dz)
                for (int dy = 0; dy < 2; ++dy)
                    for (int dxi = 0; dxi < 2; ++dxi) {
                        double wt = (double)(w[0][dxi] * w[1][dy] * w[2][dz]) * 0x1p-42;
                        double* m = s->mom[sp] + 4 * ((size_t)b * N + node_at(s, c[0] + dxi, c[1] + dy, c[2] + dz));
                        m[0] += wt; m[1] += wt * vv[0]; m[2] += wt * vv[1]; m[3] += wt * vv[2];
                        s->mke[sp][(size_t)b * N + node_at(s, c[0] + dxi, c[1] + dy, c[2] + dz)] += wt * v2;
                    }
            if (s->nfine) fine_accumulate(s, sp, p, vv);
        }
    for (size_t q = 0; q < N; ++q) s->mphi[(size_t)b * N + q] += s->phi[q];
    s->bsteps[b]++;
    s->msteps++;
}

/* ---------------------------------------------------------------------------
 * Binary Coulomb collisions (Table I, "Coulomb collision e+e, e+Ar+, Ar+ +Ar+";
 * the paper's cited binary-collision model of Takizuka and Abe, 1977), applied
 * once per step to the particles alive at its end, cell by cell:
 *   - the particles of a cell are put in the order of the key
 *     (Philox(id, step, PUR_COUL_ORDER) word 0, then id): a random pairing that
 *     does not depend on array order;
 *   - like particles pair as (0,1), (2,3), ...; an odd count makes the first
 *     three a triplet (0,1), (1,2), (2,0), each with half the time step;
 *   - e-i: every particle of the larger group A (electrons on a tie) meets
 *     B[k mod |B|]; the density is that of the smaller group;
 *   - order inside a cell: e-e, i-i, e-i.
 * One collision of A and B with relative velocity u (|u| > 0) over dt:
 *   mu = mA mB / (mA + mB),
 *   sigma^2 = qA^2 qB^2 lnL / (8 pi eps0^2 mu^2) * n * dt / |u|^3,
 *   delta = sigma * N(0,1) = tan(Theta/2): sin Theta = 2 delta / (1 + delta^2),
 *   1 - cos Theta = 2 delta^2 / (1 + delta^2), azimuth Phi from a uniform point
 *   (a, b) of the unit disk: cos Phi = (a^2 - b^2)/s, sin Phi = 2ab/s;
 *   u' = u rotated by (Theta, Phi) about the frame of u, Du = u' - u,
 *   vA += (mu/mA) Du, vB -= (mu/mB) Du  (momentum and energy are conserved).
 * Random numbers: the stream (id of the pair's first particle, step, purpose). */
static void coul_pair(double* va, double* vb, double ma, double mb, double cfac, double n, double dt, uint32_t id,
                      uint32_t step, uint32_t purpose, const uint32_t key[2])
{
    const double u[3] = { va[0] - vb[0], va[1] - vb[1], va[2] - vb[2] };
    const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (!(u2 > 0.0)) return;
    const double um = sqrt(u2);
    const double sig2 = ((cfac * n) * dt) / (u2 * um);
    rstream r; rs_init(&r, id, step, purpose, key);
    double g, g2;
    rs_gauss2(&r, &g, &g2);
    const double d = sqrt(sig2) * g;
    const double den = 1.0 + d * d;
    const double sn = (2.0 * d) / den, omc = (2.0 * (d * d)) / den;
    double a = 0.0, b = 0.0, s2 = 0.0;
    int t;
    for (t = 0; t < 128; ++t) {
        rs_pair(&r, &a, &b);
        s2 = a * a + b * b;
        if (s2 < 1.0 && s2 > 0.0) break;
    }
    double cp = 1.0, sp = 0.0;
    if (t < 128) { cp = (a * a - b * b) / s2; sp = (2.0 * (a * b)) / s2; }
    const double up = sqrt(u[0] * u[0] + u[1] * u[1]);
    double du[3];
    if (up > 0.0) {
        du[0] = (u[0] / up) * u[2] * sn * cp - (u[1] / up) * um * sn * sp - u[0] * omc;
        du[1] = (u[1] / up) * u[2] * sn * cp + (u[0] / up) * um * sn * sp - u[1] * omc;
        du[2] = -up * sn * cp - u[2] * omc;
    } else {
        du[0] = um * sn * cp;
        du[1] = um * sn * sp;
        du[2] = -u[2] * omc;
    }
    const double mu = (ma * mb) / (ma + mb);
    const double fa = mu / ma, fb = mu / mb;
    for (int q = 0; q < 3; ++q) { va[q] = va[q] + fa * du[q]; vb[q] = vb[q] - fb * du[q]; }
}

typedef struct { uint64_t key; int64_t idx; } coul_ent;
static int cmp_coul(const void* a, const void* b)
{
    const uint64_t x = ((const coul_ent*)a)->key, y = ((const coul_ent*)b)->key;
    return x < y ? -1 : (x > y ? 1 : 0);
}

void orc_coulomb(orc_sim* s)
{
    const size_t nc = cells_of(s);
    const double vol = s->c.dx * s->c.dx * s->c.dx;
    const double w = s->c.weight, lnl = s->c.coulomb_log, dt = s->c.dt;
    const uint32_t step = (uint32_t)s->step;
    const double m[2] = { ME, MAR };
    /* qA^2 qB^2 lnL / (8 pi eps0^2 mu^2) for e-e, i-i, e-i */
    double cf[3];
    for (int k = 0; k < 3; ++k) {
        const double ma = k == 1 ? MAR : ME, mb = k == 0 ? ME : MAR;
        const double mu = (ma * mb) / (ma + mb);
        cf[k] = ((((QE * QE) * (QE * QE)) * lnl) / (((8.0 * PI_D) * (EPS0 * EPS0)) * (mu * mu)));
    }
    /* particles of each species grouped by cell, in key order inside a cell */
    coul_ent* ent[2];
    size_t* start[2];
    for (int sp = 0; sp < 2; ++sp) {
        ent[sp] = (coul_ent*)malloc(sizeof(coul_ent) * (size_t)(s->n[sp] + 1));
        start[sp] = (size_t*)calloc(nc + 1, sizeof(size_t));
        int64_t* cellof = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s->n[sp] + 1));
        for (int64_t q = 0; q < s->n[sp]; ++q) {
            int c[3]; double f[3];
            locate(s, s->x[sp] + 3 * q, c, f);
            cellof[q] = (int64_t)cell_index(s, c);
            start[sp][cellof[q] + 1]++;
        }
        for (size_t c = 0; c < nc; ++c) start[sp][c + 1] += start[sp][c];
        size_t* fill = (size_t*)malloc(sizeof(size_t) * (nc + 1));
        memcpy(fill, start[sp], sizeof(size_t) * (nc + 1));
        for (int64_t q = 0; q < s->n[sp]; ++q) {
            const uint32_t id = s->id[sp][q];
            const uint32_t ctr[4] = { id, step, PUR_COUL_ORDER, 0 };
            uint32_t o[4];
            orc_philox4x32_10(ctr, s->key, o);
            coul_ent e; e.key = ((uint64_t)o[0] << 32) | id; e.idx = q;
            ent[sp][fill[cellof[q]]++] = e;
        }
        for (size_t c = 0; c < nc; ++c)
            qsort(ent[sp] + start[sp][c], start[sp][c + 1] - start[sp][c], sizeof(coul_ent), cmp_coul);
        free(fill);
        free(cellof);
    }
    for (size_t c = 0; c < nc; ++c) {
        const int64_t n0 = (int64_t)(start[0][c + 1] - start[0][c]), n1 = (int64_t)(start[1][c + 1] - start[1][c]);
        const coul_ent* E = ent[0] + start[0][c];
        const coul_ent* I = ent[1] + start[1][c];
        /* like particles */
        for (int sp = 0; sp < 2; ++sp) {
            const int64_t n = sp == 0 ? n0 : n1;
            const coul_ent* L = sp == 0 ? E : I;
            if (n < 2) continue;
            const double dens = ((double)n * w) / vol;
            double* v = s->v[sp];
            const uint32_t pur = sp == 0 ? PUR_COUL_EE : PUR_COUL_II;
            int64_t j = 0;
            if (n % 2 == 1) {
                const double h = 0.5 * dt;
                for (int t = 0; t < 3; ++t) {
                    const int64_t a = L[t].idx, b = L[(t + 1) % 3].idx;
                    coul_pair(v + 3 * a, v + 3 * b, m[sp], m[sp], cf[sp], dens, h, s->id[sp][a], step, pur, s->key);
                }
                j = 3;
            }
            for (; j + 1 < n; j += 2) {
                const int64_t a = L[j].idx, b = L[j + 1].idx;
                coul_pair(v + 3 * a, v + 3 * b, m[sp], m[sp], cf[sp], dens, dt, s->id[sp][a], step, pur, s->key);
            }
        }
        /* electrons and ions */
        if (n0 > 0 && n1 > 0) {
            const int big = n0 >= n1 ? 0 : 1;
            const int64_t na = big == 0 ? n0 : n1, nb = big == 0 ? n1 : n0;
            const coul_ent* A = big == 0 ? E : I;
            const coul_ent* B = big == 0 ? I : E;
            const double dens = ((double)nb * w) / vol;
            for (int64_t k = 0; k < na; ++k) {
                const int64_t a = A[k].idx, b = B[k % nb].idx;
                double* va = s->v[big] + 3 * a;
                double* vb = s->v[1 - big] + 3 * b;
                coul_pair(va, vb, m[big], m[1 - big], cf[2], dens, dt, s->id[big][a], step, PUR_COUL_EI, s->key);
            }
        }
    }
    for (int sp = 0; sp < 2; ++sp) { free(ent[sp]); free(start[sp]); }
}

/* Electron energy histogram (for the EEPF of Sec. IV.A): after a step's
 * collisions, each electron adds one count to (its cell plane k, bin
 * floor(eps / de)), eps = (m_e/2) |v|^2 / e in eV; energies beyond the last bin
 * go to an overflow bin. */
static void eepf_accumulate(orc_sim* s)
{
    const int nb = s->c.eepf_bins;
    const double de = s->c.eepf_de_ev;
    for (int64_t q = 0; q < s->n[0]; ++q) {
        const double* v = s->v[0] + 3 * q;
        int c[3]; double f[3];
        locate(s, s->x[0] + 3 * q, c, f);
        const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        const double eps = v2 * s->hm[0];
        const double t = eps / de;
        const int b = t < (double)nb ? (int)t : nb;
        s->eepf[(size_t)c[2] * (size_t)(nb + 1) + (size_t)b]++;
    }
    s->eepf_steps++;
}

int64_t orc_get_eepf(const orc_sim* s, int64_t* counts)
{
    if (!s->eepf) return 0;
    memcpy(counts, s->eepf, sizeof(int64_t) * (size_t)s->c.nz * (size_t)(s->c.eepf_bins + 1));
    return s->eepf_steps;
}

int orc_advance(orc_sim* s)
{
    const size_t N = nodes_of(s);
    orc_efield(s->c.nx, s->c.ny, s->c.nz, s->c.dx, s->phi, s->ex, s->ey, s->ez);
    s->nch = 0;
    const int M = s->c.md_sub > 0 ? s->c.md_sub : 1;
    const double dt = s->c.dt;
    const double dtm = dt / (double)M;
    /* particles are independent within a step: OpenMP threads take ranges of
     * them, each with its own counters and product list; survivors are then
     * compacted in their original order, so nothing depends on the threads */
    const int nt = orc_threads();
    step_log* T = (step_log*)calloc((size_t)nt, sizeof(step_log));
    for (int sp = 0; sp < 2; ++sp) {
        if (sp == 1 && (s->c.flags & ORC_IONS_FROZEN)) continue;
        const double qmdt = s->qm[sp] * dt;
        const double qmdtm = s->qm[sp] * dtm;
        const int64_t n = s->n[sp];
        unsigned char* keep_it = (unsigned char*)malloc((size_t)(n > 0 ? n : 1));
        #pragma omp parallel
        {
            step_log* t = &T[thread_id()];
            #pragma omp for schedule(static)
            for (int64_t q = 0; q < n; ++q) {
                double p[3], v[3];
                memcpy(p, s->x[sp] + 3 * q, sizeof p);
                memcpy(v, s->v[sp] + 3 * q, sizeof v);
                const uint32_t id = s->id[sp][q];
                int c[3]; double f[3]; int64_t w[3][2];
                locate(s, p, c, f);
                qweights(f, w);
                int fate = 0, grain = -1;
                keep_it[q] = 0;
                if (s->cell_ng[cell_index(s, c)] == 0) {
                    double E[3];
                    gather(s, s->ex, s->ey, s->ez, c, w, E);
                    for (int a = 0; a < 3; ++a) v[a] = v[a] + qmdt * E[a];
                    for (int a = 0; a < 3; ++a) p[a] = p[a] + v[a] * dt;
                    fate = boundary(s, p);
                } else {
                    for (int m = 0; m < M; ++m) {
                        double E[3];
                        if (m > 0) { locate(s, p, c, f); qweights(f, w); }
                        gather(s, s->ex, s->ey, s->ez, c, w, E);
                        md_correct(s, p, c, w, E);
                        for (int a = 0; a < 3; ++a) v[a] = v[a] + qmdtm * E[a];
                        for (int a = 0; a < 3; ++a) p[a] = p[a] + v[a] * dtm;
                        fate = boundary(s, p);
                        if (fate) break;
                        grain = absorbed_by(s, p);
                        if (grain >= 0) break;
                    }
                }
                if (fate == 1) { t->cnt[sp == 0 ? ORC_C_LOST_BOT_E : ORC_C_LOST_BOT_I]++; continue; }
                if (fate == 2) { t->cnt[sp == 0 ? ORC_C_LOST_TOP_E : ORC_C_LOST_TOP_I]++; continue; }
                if (fate == 3) { t->cnt[ORC_C_ERR]++; continue; }
                if (grain >= 0) {
                    #pragma omp atomic
                    s->gabs[2 * grain + sp]++;
                    t->cnt[sp == 0 ? ORC_C_ABS_E : ORC_C_ABS_I]++;
                    continue;
                }
                if (!(s->c.flags & ORC_NO_MCC)) mcc(s, t, sp, p, v, id);
                memcpy(s->x[sp] + 3 * q, p, sizeof p);
                memcpy(s->v[sp] + 3 * q, v, sizeof v);
                keep_it[q] = 1;
            }
        }
        int64_t keep = 0;
        for (int64_t q = 0; q < n; ++q) {
            if (!keep_it[q]) continue;
            if (keep != q) {
                memcpy(s->x[sp] + 3 * keep, s->x[sp] + 3 * q, 3 * sizeof(double));
                memcpy(s->v[sp] + 3 * keep, s->v[sp] + 3 * q, 3 * sizeof(double));
                s->id[sp][keep] = s->id[sp][q];
            }
            keep++;
        }
        free(keep_it);
        s->n[sp] = keep;
    }
    for (int t = 0; t < nt; ++t) {
        for (int a = 0; a < ORC_C_N; ++a) s->cnt[a] += T[t].cnt[a];
        for (int64_t r = 0; r < T[t].nch; ++r) {
            if (s->nch == s->capch) {
                s->capch = s->capch ? 2 * s->capch : 64;
                s->ch = (child_rec*)realloc(s->ch, sizeof(child_rec) * s->capch);
            }
            s->ch[s->nch++] = T[t].ch[r];
        }
        free(T[t].ch);
    }
    free(T);
    /* grain charges after this step's absorptions */
    for (int g = 0; g < s->c.n_grains; ++g)
        s->gq[g] = (QE * s->c.weight) * (double)(s->gabs[2 * g + 1] - s->gabs[2 * g + 0]);
    /* ionization products, numbered in the order of their parents' ids */
    qsort(s->ch, (size_t)s->nch, sizeof(child_rec), cmp_child);
    if ((uint64_t)s->next_id + 2u * (uint64_t)s->nch > 0xFFFFFFFFull) s->cnt[ORC_C_ERR]++;
    grow(s, 0, s->n[0] + s->nch);
    grow(s, 1, s->n[1] + s->nch);
    for (int64_t r = 0; r < s->nch; ++r) {
        const child_rec* cr = &s->ch[r];
        memcpy(s->x[0] + 3 * s->n[0], cr->x, sizeof cr->x);
        memcpy(s->v[0] + 3 * s->n[0], cr->ve, sizeof cr->ve);
        s->id[0][s->n[0]++] = s->next_id + (uint32_t)(2 * r);
        memcpy(s->x[1] + 3 * s->n[1], cr->x, sizeof cr->x);
        memcpy(s->v[1] + 3 * s->n[1], cr->vi, sizeof cr->vi);
        s->id[1][s->n[1]++] = s->next_id + (uint32_t)(2 * r + 1);
    }
    s->next_id += (uint32_t)(2 * s->nch);
    if (s->c.flags & ORC_COULOMB) orc_coulomb(s);
    if ((s->c.flags & ORC_EEPF) && s->eepf) eepf_accumulate(s);
    deposit_all(s);
    s->step++;
    (void)N;
    return 0;
}

int orc_step(orc_sim* s)
{
    int rc = orc_advance(s);
    if (rc) return rc;
    rc = orc_solve(s);
    if (rc) return rc;
    if (s->c.flags & ORC_MOMENTS) moments_accumulate(s);
    return 0;
}

/* Unit-charge mesh field of grain g on the 4x4x4 nodes of its MD region
 * (Eq. 5: E_PIC^dust per coulomb of grain charge): the exact solution of the
 * discrete Poisson equation (Eq. 3) with grounded electrodes for one coulomb
 * deposited by CIC at the grain centre, then E by the differences of Eq. 4.
 * It is the same discrete solution orc_poisson gives for that source,
 * evaluated only where the region's differences need it: the source sits on
 * 8 nodes, so each Fourier mode's right-hand side is a sum of 8 terms; one
 * tridiagonal solve per mode; the inverse transform is summed on the 6x6x6
 * nodes around the region (clipped to the electrode planes, where phi = 0).
 * tab: [(lk*4 + lj)*4 + li][3], region node (gc - 1 + (li, lj, lk)). */
static void grain_table(const orc_sim* s, int g, double* tab)
{
    const int nx = s->c.nx, ny = s->c.ny, nz = s->c.nz, P = nx * ny;
    const double dx = s->c.dx;
    const double scale1 = ((1.0 / (dx * dx * dx)) * 0x1p-42) / EPS0;
    int gc[3]; double fr[3]; int64_t w[3][2];
    locate(s, s->gpos + 3 * g, gc, fr);
    qweights(fr, w);
    double* cx = (double*)malloc(sizeof(double) * nx);
    double* sx = (double*)malloc(sizeof(double) * nx);
    double* cy = (double*)malloc(sizeof(double) * ny);
    double* sy = (double*)malloc(sizeof(double) * ny);
    double* cp = (double*)malloc(sizeof(double) * (nz + 1));
    double* rr = (double*)malloc(sizeof(double) * (nz + 1));
    double* ri = (double*)malloc(sizeof(double) * (nz + 1));
    for (int t = 0; t < nx; ++t) { cx[t] = cos(2.0 * PI_D * t / nx); sx[t] = sin(2.0 * PI_D * t / nx); }
    for (int t = 0; t < ny; ++t) { cy[t] = cos(2.0 * PI_D * t / ny); sy[t] = sin(2.0 * PI_D * t / ny); }
    /* the 6x6x6 block of nodes gc - 2 .. gc + 3: phi summed over the modes */
    double blk[6][6][6];
    memset(blk, 0, sizeof blk);
    for (int p = 0; p < P; ++p) {
        const int m1 = p % nx, m2 = p / nx;
        for (int k = 0; k <= nz; ++k) { rr[k] = 0.0; ri[k] = 0.0; }
        /* forward transform of the right-hand side -dx^2 f of the 8 source nodes */
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int di = 0; di < 2; ++di) {
                    const int i = (gc[0] + di) % nx, j = (gc[1] + dy) % ny, k = gc[2] + dz;
                    const double v = -(dx * dx) * ((double)(w[0][di] * w[1][dy] * w[2][dz]) * scale1);
                    const int t1 = (int)(((long)m1 * i) % nx), t2 = (int)(((long)m2 * j) % ny);
                    const double er = cx[t1] * cy[t2] - sx[t1] * sy[t2];     /* cos(a + b) */
                    const double ei = -(sx[t1] * cy[t2] + cx[t1] * sy[t2]);  /* -sin(a + b) */
                    rr[k] += v * er;
                    ri[k] += v * ei;
                }
        thomas_mode(nz - 1, (2.0 * cx[m1] + 2.0 * cy[m2]) - 6.0, rr, ri, cp);
        /* inverse transform at the block nodes (interior planes only) */
        for (int b = 0; b < 6; ++b) {
            const int k = gc[2] - 2 + b;
            if (k < 1 || k > nz - 1) continue;
            for (int bj = 0; bj < 6; ++bj) {
                const int j = ((gc[1] - 2 + bj) % ny + ny) % ny;
                const int t2 = (int)(((long)m2 * j) % ny);
                for (int bi = 0; bi < 6; ++bi) {
                    const int i = ((gc[0] - 2 + bi) % nx + nx) % nx;
                    const int t1 = (int)(((long)m1 * i) % nx);
                    const double er = cx[t1] * cy[t2] - sx[t1] * sy[t2];
                    const double ei = sx[t1] * cy[t2] + cx[t1] * sy[t2];
                    blk[b][bj][bi] += rr[k] * er - ri[k] * ei;
                }
            }
        }
    }
    for (int b = 0; b < 6; ++b)
        for (int bj = 0; bj < 6; ++bj)
            for (int bi = 0; bi < 6; ++bi) blk[b][bj][bi] = blk[b][bj][bi] / (double)P;
    /* E = -grad phi at the region nodes (orc_efield's formulas) */
    const double h2 = 2.0 * dx;
    for (int lk = 0; lk < 4; ++lk)
        for (int lj = 0; lj < 4; ++lj)
            for (int li = 0; li < 4; ++li) {
                const int bi = li + 1, bj = lj + 1, b = lk + 1, k = gc[2] - 1 + lk;
                double* tv = tab + ((lk * 4 + lj) * 4 + li) * 3;
                tv[0] = (blk[b][bj][bi - 1] - blk[b][bj][bi + 1]) / h2;
                tv[1] = (blk[b][bj - 1][bi] - blk[b][bj + 1][bi]) / h2;
                if (k == 0)
                    tv[2] = ((3.0 * blk[b][bj][bi] - 4.0 * blk[b + 1][bj][bi]) + blk[b + 2][bj][bi]) / h2;
                else if (k == nz)
                    tv[2] = ((4.0 * blk[b - 1][bj][bi] - 3.0 * blk[b][bj][bi]) - blk[b - 2][bj][bi]) / h2;
                else
                    tv[2] = (blk[b - 1][bj][bi] - blk[b + 1][bj][bi]) / h2;
            }
    free(cx); free(sx); free(cy); free(sy); free(cp); free(rr); free(ri);
}

/* Initial plasma drawn from the run's seed (the paper starts from a uniform
 * plasma of given density and temperatures, Sec. III; the draw itself is this
 * build's reading): particle id p takes three uniforms at a time from its
 * stream (p, step 0, PUR_INIT_POS) for a point u L in the box until the point
 * lies farther than 1.5 radii from every grain (minimum image in x and y; at
 * most 64 tries, else the last point), and three normals from (p, 0,
 * PUR_INIT_VEL) times the thermal speed sqrt(T e / m) for its velocity. */
static void sample_plasma(orc_sim* s, int sp, int64_t n, uint32_t id0, double t_ev)
{
    const double m = sp == 0 ? ME : MAR;
    const double vth = sqrt((t_ev * QE) / m);
    const double L[3] = { s->Lx, s->Ly, s->Lz };
    for (int64_t q = 0; q < n; ++q) {
        const uint32_t id = id0 + (uint32_t)q;
        double* x = s->x[sp] + 3 * q;
        rstream rp; rs_init(&rp, id, 0, PUR_INIT_POS, s->key);
        for (int t = 0; t < 64; ++t) {
            for (int a = 0; a < 3; ++a) x[a] = u01(rs_next(&rp)) * L[a];
            int near = 0;
            for (int g = 0; g < s->c.n_grains && !near; ++g) {
                double d[3];
                for (int a = 0; a < 3; ++a) {
                    d[a] = x[a] - s->gpos[3 * g + a];
                    if (a < 2 && d[a] > 0.5 * L[a]) d[a] = d[a] - L[a];
                    else if (a < 2 && d[a] < -0.5 * L[a]) d[a] = d[a] + L[a];
                }
                const double rx = 1.5 * s->grad[g];
                near = ((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]) <= rx * rx;
            }
            if (!near) break;
        }
        double nv[3];
        rstream rv; rs_init(&rv, id, 0, PUR_INIT_VEL, s->key); rs_gauss3(&rv, nv);
        for (int a = 0; a < 3; ++a) s->v[sp][3 * q + a] = vth * nv[a];
        s->id[sp][q] = id;
    }
}

orc_sim* orc_create(const orc_cfg* cfg)
{
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->c = *cfg;
    const double dx = cfg->dx;
    s->Lx = cfg->nx * dx; s->Ly = cfg->ny * dx; s->Lz = cfg->nz * dx;
    s->qm[0] = -QE / ME; s->qm[1] = QE / MAR;
    s->hm[0] = (0.5 * ME) / QE; s->hm[1] = (0.5 * MAR) / QE;
    s->pnull[0] = 1.0 - exp(-cfg->nu_max_e * cfg->dt);
    s->pnull[1] = 1.0 - exp(-cfg->nu_max_i * cfg->dt);
    s->key[0] = (uint32_t)cfg->seed ^ cfg->run_id;
    s->key[1] = (uint32_t)(cfg->seed >> 32);
    const size_t N = nodes_of(s), C = cells_of(s);
    s->rq = (int64_t*)calloc(N, sizeof(int64_t));
    s->phi = (double*)calloc(N, sizeof(double));
    s->ex = (double*)calloc(N, sizeof(double));
    s->ey = (double*)calloc(N, sizeof(double));
    s->ez = (double*)calloc(N, sizeof(double));
    s->nph = cfg->mom_phases > 1 ? cfg->mom_phases : 1;
    s->mom[0] = (double*)calloc(4 * N * (size_t)s->nph, sizeof(double));
    s->mom[1] = (double*)calloc(4 * N * (size_t)s->nph, sizeof(double));
    s->mphi = (double*)calloc(N * (size_t)s->nph, sizeof(double));
    s->mke[0] = (double*)calloc(N * (size_t)s->nph, sizeof(double));
    s->mke[1] = (double*)calloc(N * (size_t)s->nph, sizeof(double));
    s->bsteps = (int64_t*)calloc((size_t)s->nph, sizeof(int64_t));
    if (cfg->fine_n[0] > 0 && cfg->fine_n[1] > 0 && cfg->fine_n[2] > 0 && cfg->fine_h > 0.0) {
        s->nfine = (size_t)cfg->fine_n[0] * (size_t)cfg->fine_n[1] * (size_t)cfg->fine_n[2];
        s->fine[0] = (double*)calloc(4 * s->nfine, sizeof(double));
        s->fine[1] = (double*)calloc(4 * s->nfine, sizeof(double));
    }
    if ((cfg->flags & ORC_EEPF) && cfg->eepf_bins > 0 && cfg->eepf_de_ev > 0.0)
        s->eepf = (int64_t*)calloc((size_t)cfg->nz * (size_t)(cfg->eepf_bins + 1), sizeof(int64_t));
    if (cfg->n_xs > 0) {
        s->xs = (double*)malloc(sizeof(double) * 5 * cfg->n_xs);
        memcpy(s->xs, cfg->xs, sizeof(double) * 5 * cfg->n_xs);
    }
    const int ng = cfg->n_grains;
    s->gpos = (double*)calloc(3 * (ng + 1), sizeof(double));
    s->grad = (double*)calloc(ng + 1, sizeof(double));
    s->gq = (double*)calloc(ng + 1, sizeof(double));
    s->gabs = (int64_t*)calloc(2 * (ng + 1), sizeof(int64_t));
    s->gtab = (double*)calloc((size_t)(ng + 1) * 64 * 3, sizeof(double));
    if (ng) { memcpy(s->gpos, cfg->gpos, sizeof(double) * 3 * ng); memcpy(s->grad, cfg->grad, sizeof(double) * ng); }
    s->cell_ng = (int*)calloc(C, sizeof(int));
    s->cell_g = (int*)calloc(C * MAXG, sizeof(int));
    /* MD regions: each grain's cell and its 26 direct neighbours */
    for (int g = 0; g < ng; ++g) {
        const int gc[3] = { (int)floor(s->gpos[3 * g] / dx), (int)floor(s->gpos[3 * g + 1] / dx),
                            (int)floor(s->gpos[3 * g + 2] / dx) };
        for (int dk = -1; dk <= 1; ++dk)
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    int c[3] = { (gc[0] + di + cfg->nx) % cfg->nx, (gc[1] + dj + cfg->ny) % cfg->ny, gc[2] + dk };
                    if (c[2] < 0 || c[2] >= cfg->nz) continue;
                    size_t ci = cell_index(s, c);
                    if (s->cell_ng[ci] < MAXG) s->cell_g[ci * MAXG + s->cell_ng[ci]++] = g;
                    else s->cnt[ORC_C_ERR]++;
                }
    }
    /* unit-charge mesh field of each grain on the 4x4x4 nodes of its region;
     * grains are independent (one thread per grain, so the rounding does not
     * depend on the thread count) */
    #pragma omp parallel for schedule(dynamic, 1)
    for (int g = 0; g < ng; ++g) grain_table(s, g, s->gtab + (size_t)g * 64 * 3);
    uint32_t maxid = 0; int any = 0;
    for (int sp = 0; sp < 2; ++sp) {
        grow(s, sp, cfg->n_init[sp] > 0 ? cfg->n_init[sp] : 1);
        s->n[sp] = cfg->n_init[sp];
        if (cfg->n_init[sp] > 0 && !cfg->x_init[sp]) {
            sample_plasma(s, sp, cfg->n_init[sp], sp == 0 ? 0u : (uint32_t)cfg->n_init[0], cfg->t_init_ev[sp]);
            for (int64_t q = 0; q < cfg->n_init[sp]; ++q)
                if (!any || s->id[sp][q] > maxid) { maxid = s->id[sp][q]; any = 1; }
        } else if (cfg->n_init[sp] > 0) {
            memcpy(s->x[sp], cfg->x_init[sp], sizeof(double) * 3 * cfg->n_init[sp]);
            memcpy(s->v[sp], cfg->v_init[sp], sizeof(double) * 3 * cfg->n_init[sp]);
            memcpy(s->id[sp], cfg->id_init[sp], sizeof(uint32_t) * cfg->n_init[sp]);
            for (int64_t q = 0; q < cfg->n_init[sp]; ++q)
                if (!any || s->id[sp][q] > maxid) { maxid = s->id[sp][q]; any = 1; }
        }
    }
    s->next_id = any ? maxid + 1 : 0;
    s->step = 0;
    deposit_all(s);
    orc_solve(s);
    return s;
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    for (int sp = 0; sp < 2; ++sp) { free(s->x[sp]); free(s->v[sp]); free(s->id[sp]); free(s->mom[sp]); }
    free(s->rq); free(s->phi); free(s->ex); free(s->ey); free(s->ez); free(s->xs);
    free(s->gpos); free(s->grad); free(s->gq); free(s->gabs); free(s->gtab);
    free(s->cell_ng); free(s->cell_g); free(s->ch); free(s->mphi); free(s->eepf);
    free(s->bsteps); free(s->fine[0]); free(s->fine[1]); free(s->mke[0]); free(s->mke[1]);
    free(s);
}

int64_t orc_count(const orc_sim* s, int sp) { return s->n[sp]; }
void orc_get_particles(const orc_sim* s, int sp, double* x, double* v, uint32_t* id)
{
    memcpy(x, s->x[sp], sizeof(double) * 3 * s->n[sp]);
    memcpy(v, s->v[sp], sizeof(double) * 3 * s->n[sp]);
    memcpy(id, s->id[sp], sizeof(uint32_t) * s->n[sp]);
}
void orc_get_rho(const orc_sim* s, int64_t* rq) { memcpy(rq, s->rq, sizeof(int64_t) * nodes_of(s)); }
void orc_get_phi(const orc_sim* s, double* phi) { memcpy(phi, s->phi, sizeof(double) * nodes_of(s)); }
void orc_set_phi(orc_sim* s, const double* phi) { memcpy(s->phi, phi, sizeof(double) * nodes_of(s)); }
void orc_get_grains(const orc_sim* s, int64_t* n_abs, double* q)
{
    memcpy(n_abs, s->gabs, sizeof(int64_t) * 2 * s->c.n_grains);
    memcpy(q, s->gq, sizeof(double) * s->c.n_grains);
}
void orc_get_gtab(const orc_sim* s, double* tab) { memcpy(tab, s->gtab, sizeof(double) * 64 * 3 * s->c.n_grains); }
void orc_set_gtab(orc_sim* s, const double* tab) { memcpy(s->gtab, tab, sizeof(double) * 64 * 3 * s->c.n_grains); }
void orc_get_counters(const orc_sim* s, int64_t* c) { memcpy(c, s->cnt, sizeof(int64_t) * ORC_C_N); }
int64_t orc_step_index(const orc_sim* s) { return s->step; }
uint32_t orc_next_id(const orc_sim* s) { return s->next_id; }

/* window sums of bins [b0, b1) at node q for species sp: count, count v, count |v|^2 */
static void node_sums(const orc_sim* s, int sp, int b0, int b1, size_t q, double out[5])
{
    const size_t N = nodes_of(s);
    for (int a = 0; a < 5; ++a) out[a] = 0.0;
    for (int b = b0; b < b1; ++b) {
        const double* m = s->mom[sp] + 4 * ((size_t)b * N + q);
        for (int a = 0; a < 4; ++a) out[a] += m[a];
        out[4] += s->mke[sp][(size_t)b * N + q];
    }
}

/* temperature (eV) of a species from window sums: (m / 3e) (<v^2> - |<v>|^2) */
static double temperature(const double sum[5], double m)
{
    if (!(sum[0] > 0.0)) return 0.0;
    const double u[3] = { sum[1] / sum[0], sum[2] / sum[0], sum[3] / sum[0] };
    const double var = sum[4] / sum[0] - ((u[0] * u[0] + u[1] * u[1]) + u[2] * u[2]);
    return (m / (3.0 * QE)) * var;
}

/* window averages of bins [b0, b1): sums over the bins' samples divided by their count */
static int moments_of(const orc_sim* s, int what, int b0, int b1, int64_t steps, double* out)
{
    const size_t N = nodes_of(s);
    if (steps == 0 || what < 0 || what > 6) return -1;
    if (what >= 5) {
        const int sp = what - 5;
        for (size_t q = 0; q < N; ++q) {
            double sum[5];
            node_sums(s, sp, b0, b1, q, sum);
            out[q] = temperature(sum, sp == 0 ? ME : MAR);
        }
        return 0;
    }
    const double dx = s->c.dx;
    const double norm = s->c.weight / ((dx * dx * dx) * (double)steps);
    const size_t len = what >= 3 ? 3 * N : N;
    for (size_t q = 0; q < len; ++q) out[q] = 0.0;
    for (int b = b0; b < b1; ++b) {
        if (what == 0) {
            for (size_t q = 0; q < N; ++q) out[q] += s->mphi[(size_t)b * N + q];
        } else {
            const double* m = s->mom[(what - 1) % 2] + 4 * (size_t)b * N;
            for (size_t q = 0; q < N; ++q) {
                if (what <= 2) out[q] += m[4 * q];
                else
                    for (int a = 0; a < 3; ++a) out[3 * q + a] += m[4 * q + 1 + a];
            }
        }
    }
    const double scale = what == 0 ? 1.0 / (double)steps : norm;
    for (size_t q = 0; q < len; ++q) out[q] *= scale;
    return 0;
}

/* ---------------------------------------------------------------------------
 * Hypothetical grain charge from local plasma moments (Sec. IV.B: the charge a
 * grain would carry with no other grains around, from the orbital-motion-
 * limited balance of electron and ion fluxes including the charge-exchange ion
 * flux, with the local densities and temperatures).  Currents per pi a^2 with
 * the mean speeds vbar_s = sqrt(8 e T_s / (pi m_s)):
 *   phi <= 0:  J_e = n_e vbar_e exp(phi/T_e),
 *              J_i = n_i vbar_i (1 - phi/T_i + 0.1 (phi/T_i)^2 lambda_D/l_i)
 *   phi >  0:  J_e = n_e vbar_e (1 + phi/T_e),  J_i = n_i vbar_i exp(-phi/T_i)
 * (the quadratic term is the weakly collisional charge-exchange correction of
 * Khrapak et al., Phys. Rev. E 72, 016406 (2005)); J_e - J_i increases with
 * phi and has one root, found here by bisection. */
double orc_oml_potential(double ne, double ni, double te, double ti, double lam_over_l)
{
    if (!(ne > 0.0) || !(ni > 0.0) || !(te > 0.0) || !(ti > 0.0)) return NAN;
    const double ve = sqrt((8.0 * QE * te) / (PI_D * ME));
    const double vi = sqrt((8.0 * QE * ti) / (PI_D * MAR));
    const double A = (ne * ve) / (ni * vi);
    double lo, hi;
    if (A > 1.0) { lo = -200.0 * te; hi = 0.0; }
    else if (A < 1.0) { lo = 0.0; hi = 200.0 * ti; }
    else return 0.0;
    for (int it = 0; it < 400; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double f;
        if (mid <= 0.0) {
            const double x = mid / ti;
            f = A * exp(mid / te) - (1.0 - x + 0.1 * x * x * lam_over_l);
        } else {
            f = A * (1.0 + mid / te) - exp(-mid / ti);
        }
        if (f > 0.0) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

int orc_oml_charges(const orc_sim* s, int with_cx, double* out)
{
    if (s->msteps == 0) return -1;
    const double dx = s->c.dx;
    const double norm = s->c.weight / ((dx * dx * dx) * (double)s->msteps);
    for (int g = 0; g < s->c.n_grains; ++g) {
        const double* p = s->gpos + 3 * g;
        int c[3]; double f[3];
        locate(s, p, c, f);
        double sum[2][5] = {{0}};
        for (int dz = 0; dz < 2; ++dz)
            for (int dy = 0; dy < 2; ++dy)
                for (int dxi = 0; dxi < 2; ++dxi) {
                    const double w = (dxi ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                    const size_t q = node_at(s, c[0] + dxi, c[1] + dy, c[2] + dz);
                    for (int sp = 0; sp < 2; ++sp) {
                        double ns[5];
                        node_sums(s, sp, 0, s->nph, q, ns);
                        for (int a = 0; a < 5; ++a) sum[sp][a] += w * ns[a];
                    }
                }
        const double ne = sum[0][0] * norm, ni = sum[1][0] * norm;
        const double te = temperature(sum[0], ME), ti = temperature(sum[1], MAR);
        double lam_l = 0.0;
        if (with_cx && ne > 0.0 && ni > 0.0 && te > 0.0 && ti > 0.0 && s->c.n_xs > 0) {
            const double lde2 = (EPS0 * te) / (ne * QE), ldi2 = (EPS0 * ti) / (ni * QE);
            const double lam = 1.0 / sqrt(1.0 / lde2 + 1.0 / ldi2);
            const double sig = xs_at(s->xs + 4 * s->c.n_xs, s->c.n_xs, s->c.de_i, 1.5 * ti);
            lam_l = lam * (s->c.n_gas * sig);
        }
        const double phi = orc_oml_potential(ne, ni, te, ti, lam_l);
        double* o = out + 6 * g;
        o[0] = 4.0 * PI_D * EPS0 * s->grad[g] * phi;
        o[1] = phi; o[2] = ne; o[3] = ni; o[4] = te; o[5] = ti;
    }
    return 0;
}

int orc_moments(const orc_sim* s, int what, double* out)
{
    return moments_of(s, what, 0, s->nph, s->msteps, out);
}

int orc_moments_phase(const orc_sim* s, int what, int bin, double* out, int64_t* steps)
{
    if (bin < 0 || bin >= s->nph) return -1;
    if (steps) *steps = s->bsteps[bin];
    return moments_of(s, what, bin, bin + 1, s->bsteps[bin], out);
}

int orc_fine_moments(const orc_sim* s, int what, double* out)
{
    if (!s->nfine || s->msteps == 0 || what < 1 || what > 4) return -1;
    const double h = s->c.fine_h;
    const double norm = s->c.weight / ((h * h * h) * (double)s->msteps);
    const double* m = s->fine[(what - 1) % 2];
    for (size_t q = 0; q < s->nfine; ++q) {
        if (what <= 2) out[q] = m[4 * q] * norm;
        else
            for (int a = 0; a < 3; ++a) out[3 * q + a] = m[4 * q + 1 + a] * norm;
    }
    return 0;
}

int orc_field_at(orc_sim* s, const double p[3], double E[3])
{
    int c[3]; double f[3]; int64_t w[3][2];
    orc_efield(s->c.nx, s->c.ny, s->c.nz, s->c.dx, s->phi, s->ex, s->ey, s->ez);
    locate(s, p, c, f);
    qweights(f, w);
    gather(s, s->ex, s->ey, s->ez, c, w, E);
    int md = s->cell_ng[cell_index(s, c)] > 0;
    if (md) md_correct(s, p, c, w, E);
    return md;
}

void orc_set_grain_counts(orc_sim* s, const int64_t* n_abs)
{
    memcpy(s->gabs, n_abs, sizeof(int64_t) * 2 * s->c.n_grains);
    for (int g = 0; g < s->c.n_grains; ++g)
        s->gq[g] = (QE * s->c.weight) * (double)(s->gabs[2 * g + 1] - s->gabs[2 * g + 0]);
    deposit_all(s);
    orc_solve(s);
}

void orc_reset_moments(orc_sim* s)
{
    const size_t N = nodes_of(s) * (size_t)s->nph;
    memset(s->mom[0], 0, sizeof(double) * 4 * N);
    memset(s->mom[1], 0, sizeof(double) * 4 * N);
    memset(s->mphi, 0, sizeof(double) * N);
    memset(s->mke[0], 0, sizeof(double) * N);
    memset(s->mke[1], 0, sizeof(double) * N);
    memset(s->bsteps, 0, sizeof(int64_t) * (size_t)s->nph);
    if (s->nfine) {
        memset(s->fine[0], 0, sizeof(double) * 4 * s->nfine);
        memset(s->fine[1], 0, sizeof(double) * 4 * s->nfine);
    }
    s->msteps = 0;
}

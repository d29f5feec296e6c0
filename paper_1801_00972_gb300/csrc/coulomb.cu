// Binary Coulomb collisions e-e, e-Ar+, Ar+-Ar+ (Table I), once per step
// after the ionization products join, with the binary-collision model the
// paper cites (Sec. III): particles of a cell are paired at random, and each
// pair's relative velocity u turns by an angle Theta with tan(Theta/2) normal
// of variance q_A^2 q_B^2 lnL n dt / (8 pi eps0^2 mu^2 |u|^3) and a uniform
// azimuth; momentum and energy are conserved pair by pair.
//
//   k_coul_count   particles per cell and species (warp-aggregated atomics)
//   (exclusive scan of the counts)
//   k_coul_scatter slot indices grouped by cell, with the pairing key
//                  (Philox word of (id, step, purpose 6), then id)
//   k_coul_cells   one thread per cell: the cell's lists put in key order,
//                  then e-e, Ar+-Ar+ and e-Ar+ collisions in turn
//
// Pairing: like particles (0,1), (2,3), ...; an odd count's first three form
// the triplet (0,1), (1,2), (2,0) at half the time step.  Unlike: every
// particle of the larger group A (electrons on a tie) meets B[k mod |B|], at
// the density of B.  The random numbers of a collision come from the stream
// (id of its first particle, step, purpose 7 e-e / 8 i-i / 9 e-i).  None of
// this depends on where particles sit in the arrays.
//
// The FP64 unit is built without fused multiply-add: its arithmetic follows
// the oracle's operation for operation, so an FP64 run matches it bit for
// bit.  The mixed unit works in float, in the particles' cells/step units.
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr uint32_t kPurCoulOrder = 6, kPurCoulEE = 7, kPurCoulII = 8, kPurCoulEI = 9;

__device__ __forceinline__ int coul_cell(const float4& p, int nx, int ny)
{
    const int c = __float_as_int(p.w);   // packed i | j << 10 | k << 20, -1 dead
    if (c < 0) return -1;
    return ((c >> 20) * ny + ((c >> 10) & 1023)) * nx + (c & 1023);
}
__device__ __forceinline__ int coul_cell(const double4& p, int, int) { return p.w < 0.0 ? -1 : (int)p.w; }
__device__ __forceinline__ uint32_t coul_id(const float4& v) { return __float_as_uint(v.w); }
__device__ __forceinline__ uint32_t coul_id(const double4& v) { return (uint32_t)v.w; }

template <typename T4>
__global__ void k_coul_count(const T4* __restrict__ pos, const unsigned long long* nslot, int sp, unsigned int* cnt,
                             int nx, int ny)
{
    const unsigned long long n = nslot[sp];
    const int lane = threadIdx.x & 31;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const int c = coul_cell(pos[q], nx, ny);
        const unsigned m = __match_any_sync(__activemask(), c);
        if (c >= 0 && lane == __ffs(m) - 1) atomicAdd(cnt + c, (unsigned int)__popc(m));
    }
}

// cur holds each cell's first slot on entry and its end on exit
template <typename T4>
__global__ void k_coul_scatter(const T4* __restrict__ pos, const T4* __restrict__ vel,
                               const unsigned long long* nslot, int sp, unsigned int* cur, unsigned int* idx,
                               unsigned long long* key, int nx, int ny, const uint32_t* step, uint2 pkey)
{
    const unsigned long long n = nslot[sp];
    const uint32_t st = *step - 1u;   // the particle side of this step is complete
    const int lane = threadIdx.x & 31;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const int c = coul_cell(pos[q], nx, ny);
        const unsigned m = __match_any_sync(__activemask(), c);
        const int leader = __ffs(m) - 1;
        unsigned int base = 0;
        if (c >= 0 && lane == leader) base = atomicAdd(cur + c, (unsigned int)__popc(m));
        base = __shfl_sync(m, base, leader);
        if (c < 0) continue;
        const unsigned int d = base + (unsigned int)__popc(m & ((1u << lane) - 1u));
        const uint32_t id = coul_id(vel[q]);
        const uint4 h = philox4x32_10(make_uint4(id, st, kPurCoulOrder, 0u), pkey);
        idx[d] = (unsigned int)q;
        key[d] = ((unsigned long long)h.x << 32) | id;
    }
}

// insertion sort of one cell's entries by key
__device__ void coul_sort(unsigned long long* key, unsigned int* idx, unsigned int a, unsigned int b)
{
    for (unsigned int i = a + 1; i < b; ++i) {
        const unsigned long long k = key[i];
        const unsigned int x = idx[i];
        unsigned int j = i;
        while (j > a && key[j - 1] > k) {
            key[j] = key[j - 1];
            idx[j] = idx[j - 1];
            --j;
        }
        key[j] = k;
        idx[j] = x;
    }
}

// ---- FP64: SI units, the oracle's operations in its order -----------------
__device__ void coul_pair64(double* va, double* vb, double ma, double mb, double cfac, double n, double dt,
                            uint32_t id, uint32_t step, uint32_t purpose, uint2 pkey)
{
    const double u[3] = {va[0] - vb[0], va[1] - vb[1], va[2] - vb[2]};
    const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (!(u2 > 0.0)) return;
    const double um = sqrt(u2);
    const double sig2 = ((cfac * n) * dt) / (u2 * um);
    RStream r(id, step, purpose, pkey);
    double g = 0.0;
    for (int t = 0; t < 128; ++t) {
        const double a = 2.0 * u01d(r.next()) - 1.0;
        const double b = 2.0 * u01d(r.next()) - 1.0;
        const double s = a * a + b * b;
        if (s < 1.0) {
            g = a * sqrt((-2.0 * ln_series(s)) / s);
            break;
        }
    }
    const double d = sqrt(sig2) * g;
    const double den = 1.0 + d * d;
    const double sn = (2.0 * d) / den, omc = (2.0 * (d * d)) / den;
    double a = 0.0, b = 0.0, s2 = 0.0;
    int t;
    for (t = 0; t < 128; ++t) {
        a = 2.0 * u01d(r.next()) - 1.0;
        b = 2.0 * u01d(r.next()) - 1.0;
        s2 = a * a + b * b;
        if (s2 < 1.0 && s2 > 0.0) break;
    }
    double cp = 1.0, sp = 0.0;
    if (t < 128) {
        cp = (a * a - b * b) / s2;
        sp = (2.0 * (a * b)) / s2;
    }
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
    for (int q = 0; q < 3; ++q) {
        va[q] = va[q] + fa * du[q];
        vb[q] = vb[q] - fb * du[q];
    }
}

// ---- mixed: float, velocities in cells/step --------------------------------
__device__ void coul_pair32(float* va, float* vb, float fa, float fb, float cfac, float n, float dtf, uint32_t id,
                            uint32_t step, uint32_t purpose, uint2 pkey)
{
    const float u[3] = {va[0] - vb[0], va[1] - vb[1], va[2] - vb[2]};
    const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (!(u2 > 0.f)) return;
    const float um = sqrtf(u2);
    const float sig2 = ((cfac * n) * dtf) / (u2 * um);
    RStream r(id, step, purpose, pkey);
    float g = 0.f;
    for (int t = 0; t < 128; ++t) {
        const float a = 2.f * u01f(r.next()) - 1.f;
        const float b = 2.f * u01f(r.next()) - 1.f;
        const float s = a * a + b * b;
        if (s < 1.f && s > 0.f) {
            g = a * sqrtf(-2.f * logf(s) / s);
            break;
        }
    }
    const float d = sqrtf(sig2) * g;
    const float den = 1.f + d * d;
    const float sn = 2.f * d / den, omc = 2.f * d * d / den;
    float a = 0.f, b = 0.f, s2 = 0.f;
    int t;
    for (t = 0; t < 128; ++t) {
        a = 2.f * u01f(r.next()) - 1.f;
        b = 2.f * u01f(r.next()) - 1.f;
        s2 = a * a + b * b;
        if (s2 < 1.f && s2 > 0.f) break;
    }
    float cp = 1.f, sp = 0.f;
    if (t < 128) {
        cp = (a * a - b * b) / s2;
        sp = 2.f * a * b / s2;
    }
    const float up = sqrtf(u[0] * u[0] + u[1] * u[1]);
    float du[3];
    if (up > 0.f) {
        du[0] = (u[0] / up) * u[2] * sn * cp - (u[1] / up) * um * sn * sp - u[0] * omc;
        du[1] = (u[1] / up) * u[2] * sn * cp + (u[0] / up) * um * sn * sp - u[1] * omc;
        du[2] = -up * sn * cp - u[2] * omc;
    } else {
        du[0] = um * sn * cp;
        du[1] = um * sn * sp;
        du[2] = -u[2] * omc;
    }
    for (int q = 0; q < 3; ++q) {
        va[q] += fa * du[q];
        vb[q] -= fb * du[q];
    }
}

struct CoulArgs {
    const unsigned int* end[2];   // per species: end slot of each cell's group
    unsigned int* idx[2];
    unsigned long long* key[2];
    void* vel[2];
    int cells;
    double w, vol, dt;            // weight, cell volume, step
    double cf[3];                 // e-e, i-i, e-i: q^4 lnL / (8 pi eps0^2 mu^2) (SI); mixed: times dt / (dx/dt)^3
    double m[2];                  // masses (kg)
    const uint32_t* step;
    uint2 pkey;
};

__device__ __forceinline__ uint32_t load_v(const CoulArgs& a, int sp, unsigned int q, double v[3])
{
    const double4 x = reinterpret_cast<const double4*>(a.vel[sp])[q];
    v[0] = x.x; v[1] = x.y; v[2] = x.z;
    return (uint32_t)x.w;
}
__device__ __forceinline__ void store_v(const CoulArgs& a, int sp, unsigned int q, const double v[3])
{
    double4* p = reinterpret_cast<double4*>(a.vel[sp]) + q;
    const double w = p->w;
    *p = make_double4(v[0], v[1], v[2], w);
}
__device__ __forceinline__ uint32_t load_v(const CoulArgs& a, int sp, unsigned int q, float v[3])
{
    const float4 x = reinterpret_cast<const float4*>(a.vel[sp])[q];
    v[0] = x.x; v[1] = x.y; v[2] = x.z;
    return __float_as_uint(x.w);
}
__device__ __forceinline__ void store_v(const CoulArgs& a, int sp, unsigned int q, const float v[3])
{
    float4* p = reinterpret_cast<float4*>(a.vel[sp]) + q;
    const float w = p->w;
    *p = make_float4(v[0], v[1], v[2], w);
}

// one collision of slot qa (species sa, the pair's first particle) with slot qb
// (species sb); kind 0 e-e, 1 i-i, 2 e-i
__device__ __forceinline__ void collide(const CoulArgs& a, int sa, unsigned int qa, int sb, unsigned int qb,
                                        int kind, double dens, bool half, uint32_t step, uint32_t purpose, double*)
{
    double va[3], vb[3];
    const uint32_t ida = load_v(a, sa, qa, va);
    load_v(a, sb, qb, vb);
    const double dt = half ? 0.5 * a.dt : a.dt;
    coul_pair64(va, vb, a.m[sa], a.m[sb], a.cf[kind], dens, dt, ida, step, purpose, a.pkey);
    store_v(a, sa, qa, va);
    store_v(a, sb, qb, vb);
}
__device__ __forceinline__ void collide(const CoulArgs& a, int sa, unsigned int qa, int sb, unsigned int qb,
                                        int kind, double dens, bool half, uint32_t step, uint32_t purpose, float*)
{
    float va[3], vb[3];
    const uint32_t ida = load_v(a, sa, qa, va);
    load_v(a, sb, qb, vb);
    const double mu = (a.m[sa] * a.m[sb]) / (a.m[sa] + a.m[sb]);
    coul_pair32(va, vb, (float)(mu / a.m[sa]), (float)(mu / a.m[sb]), (float)a.cf[kind], (float)dens,
                half ? 0.5f : 1.f, ida, step, purpose, a.pkey);
    store_v(a, sa, qa, va);
    store_v(a, sb, qb, vb);
}

// Form for a cell with more than kCoulLocal particles of a species: the groups
// put in key order in place in global memory.
template <typename T>
__device__ void cell_serial(const CoulArgs& a, int c, uint32_t step)
{
    unsigned int b0[2], b1[2];
    for (int sp = 0; sp < 2; ++sp) {
        b0[sp] = c == 0 ? 0u : a.end[sp][c - 1];
        b1[sp] = a.end[sp][c];
        coul_sort(a.key[sp], a.idx[sp], b0[sp], b1[sp]);
    }
    T* tag = nullptr;
    for (int sp = 0; sp < 2; ++sp) {
        const unsigned int n = b1[sp] - b0[sp];
        if (n < 2) continue;
        const unsigned int* L = a.idx[sp] + b0[sp];
        const double dens = ((double)n * a.w) / a.vol;
        const uint32_t pur = sp == 0 ? kPurCoulEE : kPurCoulII;
        unsigned int j = 0;
        if (n % 2 == 1) {
            for (int t = 0; t < 3; ++t) collide(a, sp, L[t], sp, L[(t + 1) % 3], sp, dens, true, step, pur, tag);
            j = 3;
        }
        for (; j + 1 < n; j += 2) collide(a, sp, L[j], sp, L[j + 1], sp, dens, false, step, pur, tag);
    }
    const unsigned int ne = b1[0] - b0[0], ni = b1[1] - b0[1];
    if (ne > 0 && ni > 0) {
        const int big = ne >= ni ? 0 : 1;
        const unsigned int na = big == 0 ? ne : ni, nb = big == 0 ? ni : ne;
        const unsigned int* A = a.idx[big] + b0[big];
        const unsigned int* B = a.idx[1 - big] + b0[1 - big];
        const double dens = ((double)nb * a.w) / a.vol;
        for (unsigned int k = 0; k < na; ++k)
            collide(a, big, A[k], 1 - big, B[k % nb], 2, dens, false, step, kPurCoulEI, tag);
    }
}

// One thread per cell.  A group of at most kCoulLocal particles is put in key
// order in a local array (insertion sort on cached memory) and collided from
// there; a larger cell takes the serial form above, in place.
constexpr int kCoulLocal = 32;

template <typename T>
__global__ void __launch_bounds__(128) k_coul_cells(const CoulArgs a)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.cells) return;
    const uint32_t step = *a.step - 1u;
    unsigned int b0[2], n[2];
    for (int sp = 0; sp < 2; ++sp) {
        b0[sp] = c == 0 ? 0u : a.end[sp][c - 1];
        n[sp] = a.end[sp][c] - b0[sp];
    }
    if (n[0] + n[1] < 2) return;
    if (n[0] > kCoulLocal || n[1] > kCoulLocal) {
        cell_serial<T>(a, c, step);
        return;
    }
    unsigned int list[2][kCoulLocal];
    for (int sp = 0; sp < 2; ++sp) {
        unsigned long long key[kCoulLocal];
        for (unsigned int i = 0; i < n[sp]; ++i) {
            const unsigned long long k = a.key[sp][b0[sp] + i];
            const unsigned int q = a.idx[sp][b0[sp] + i];
            unsigned int j = i;
            while (j > 0 && key[j - 1] > k) {
                key[j] = key[j - 1];
                list[sp][j] = list[sp][j - 1];
                --j;
            }
            key[j] = k;
            list[sp][j] = q;
        }
    }
    T* tag = nullptr;
    for (int sp = 0; sp < 2; ++sp) {
        const unsigned int m = n[sp];
        if (m < 2) continue;
        const unsigned int* L = list[sp];
        const double dens = ((double)m * a.w) / a.vol;
        const uint32_t pur = sp == 0 ? kPurCoulEE : kPurCoulII;
        unsigned int j = 0;
        if (m % 2 == 1) {
            for (int t = 0; t < 3; ++t) collide(a, sp, L[t], sp, L[(t + 1) % 3], sp, dens, true, step, pur, tag);
            j = 3;
        }
        for (; j + 1 < m; j += 2) collide(a, sp, L[j], sp, L[j + 1], sp, dens, false, step, pur, tag);
    }
    if (n[0] > 0 && n[1] > 0) {
        const int big = n[0] >= n[1] ? 0 : 1;
        const unsigned int na = n[big], nb = n[1 - big];
        const unsigned int* A = list[big];
        const unsigned int* B = list[1 - big];
        const double dens = ((double)nb * a.w) / a.vol;
        for (unsigned int k = 0; k < na; ++k)
            collide(a, big, A[k], 1 - big, B[k % nb], 2, dens, false, step, kPurCoulEI, tag);
    }
}

}  // namespace

void launch_coulomb(pic_ctx* c)
{
    const bool mixed = c->prec == PIC_MIXED;
    const size_t nc = c->cells;
    CoulArgs a{};
    for (int sp = 0; sp < 2; ++sp) {
        cudaMemsetAsync(c->cs_end[sp], 0, sizeof(unsigned int) * nc, c->stream);
        const int grid = grid_for(c->cap[sp], 256, 152 * 8);
        if (mixed)
            k_coul_count<float4><<<grid, 256, 0, c->stream>>>((const float4*)c->pos[sp], c->d_nslot, sp,
                                                              c->cs_end[sp], c->nx, c->ny);
        else
            k_coul_count<double4><<<grid, 256, 0, c->stream>>>((const double4*)c->pos[sp], c->d_nslot, sp,
                                                               c->cs_end[sp], c->nx, c->ny);
        scan_cells(c, c->cs_end[sp]);
        if (mixed)
            k_coul_scatter<float4><<<grid, 256, 0, c->stream>>>((const float4*)c->pos[sp], (const float4*)c->vel[sp],
                                                                c->d_nslot, sp, c->cs_end[sp], c->cs_idx[sp],
                                                                c->cs_key[sp], c->nx, c->ny, c->d_step, c->key);
        else
            k_coul_scatter<double4><<<grid, 256, 0, c->stream>>>(
                (const double4*)c->pos[sp], (const double4*)c->vel[sp], c->d_nslot, sp, c->cs_end[sp],
                c->cs_idx[sp], c->cs_key[sp], c->nx, c->ny, c->d_step, c->key);
        c->launches += 2;
        a.end[sp] = c->cs_end[sp];
        a.idx[sp] = c->cs_idx[sp];
        a.key[sp] = c->cs_key[sp];
        a.vel[sp] = c->vel[sp];
    }
    a.cells = (int)nc;
    a.w = c->W;
    a.vol = c->dx * c->dx * c->dx;
    a.dt = c->dt;
    a.m[0] = kME;
    a.m[1] = kMAR;
    const double vs = c->dx / c->dt;
    for (int k = 0; k < 3; ++k) {
        const double ma = k == 1 ? kMAR : kME, mb = k == 0 ? kME : kMAR;
        const double mu = (ma * mb) / (ma + mb);
        const double cf = ((((kQE * kQE) * (kQE * kQE)) * c->coul_log) / (((8.0 * kPI) * (kEPS0 * kEPS0)) * (mu * mu)));
        a.cf[k] = mixed ? cf * c->dt / (vs * vs * vs) : cf;
    }
    a.step = c->d_step;
    a.pkey = c->key;
    const int grid = (int)((nc + 127) / 128);
    if (mixed) k_coul_cells<float><<<grid, 128, 0, c->stream>>>(a);
    else k_coul_cells<double><<<grid, 128, 0, c->stream>>>(a);
    c->launches += 1;
}

}  // namespace pic

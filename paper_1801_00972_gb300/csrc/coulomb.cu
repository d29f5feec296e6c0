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
//                  (Philox word of (id, step, purpose 6), then id) and the cell
//   k_coul_rank    one thread per grouped particle: its rank among its cell's
//                  keys puts the group in key order
//   k_coul_like    one thread per like pair (the triplet of an odd group on
//                  one thread, in order): e-e and Ar+-Ar+ collisions
//   k_coul_unlike  one thread per particle of the smaller group of a cell: its
//                  e-Ar+ collisions in the order of the larger group
// (both stage their work items per warp in shared memory, so that warps run full)
// Every particle meets its partners in the same order as in a cell-by-cell
// loop, so the results are those of that loop.
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
#include <algorithm>

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
                               unsigned long long* key, unsigned int* cellof, int nx, int ny, const uint32_t* step,
                               uint2 pkey)
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
        cellof[d] = (unsigned int)c;
    }
}

// The words of a collision's stream (id, step, purpose), consumed in pairs in
// the stream's order: word j is component j mod 4 of the Philox block with
// counter word j / 4.  The first two blocks are drawn up front, where every lane
// of a warp draws them together; only the few pairs that run past them (a
// collision whose rejection loops took more than four trials) draw later.
struct PairStream {
    uint4 b0, b1, ctr;
    uint2 key;
    int k;   // next pair: 0..3 in (b0, b1)
    __device__ __forceinline__ PairStream(uint32_t id, uint32_t step, uint32_t purpose, uint2 kk)
        : ctr(make_uint4(id, step, purpose, 0u)), key(kk), k(0)
    {
        b0 = philox4x32_10(ctr, key);
        ctr.w = 1u;
        b1 = philox4x32_10(ctr, key);
        ctr.w = 2u;
    }
    __device__ __forceinline__ uint2 next()
    {
        if (k == 4) {
            b0 = philox4x32_10(ctr, key);
            ctr.w += 1u;
            b1 = philox4x32_10(ctr, key);
            ctr.w += 1u;
            k = 0;
        }
        const uint2 v = k == 0 ? make_uint2(b0.x, b0.y) : k == 1 ? make_uint2(b0.z, b0.w)
                      : k == 2 ? make_uint2(b1.x, b1.y) : make_uint2(b1.z, b1.w);
        ++k;
        return v;
    }
};

// ---- FP64: SI units, the oracle's operations in its order -----------------
__device__ void coul_pair64(double* va, double* vb, double fa, double fb, double cfac, double n, double dt,
                            uint32_t id, uint32_t step, uint32_t purpose, uint2 pkey)
{
    const double u[3] = {va[0] - vb[0], va[1] - vb[1], va[2] - vb[2]};
    const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (!(u2 > 0.0)) return;
    const double um = sqrt(u2);
    const double sig2 = ((cfac * n) * dt) / (u2 * um);
    PairStream r(id, step, purpose, pkey);
    double g = 0.0;
    for (int t = 0; t < 128; ++t) {
        const uint2 w = r.next();
        const double a = 2.0 * u01d(w.x) - 1.0;
        const double b = 2.0 * u01d(w.y) - 1.0;
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
        const uint2 w = r.next();
        a = 2.0 * u01d(w.x) - 1.0;
        b = 2.0 * u01d(w.y) - 1.0;
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
    for (int q = 0; q < 3; ++q) {
        va[q] = va[q] + fa * du[q];
        vb[q] = vb[q] - fb * du[q];
    }
}

// ---- mixed: float, velocities in cells/step --------------------------------
// The same steps with reciprocals and reciprocal square roots in place of the
// divisions and square roots (a few ulp; the pass is compared with the oracle
// statistically, not bit for bit).
__device__ void coul_pair32(float* va, float* vb, float fa, float fb, float cfac, float n, float dtf, uint32_t id,
                            uint32_t step, uint32_t purpose, uint2 pkey)
{
    const float u[3] = {va[0] - vb[0], va[1] - vb[1], va[2] - vb[2]};
    const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (!(u2 > 0.f)) return;
    const float ru = rsqrtf(u2);
    const float um = u2 * ru;
    const float sig2 = ((cfac * n) * dtf) * (ru * ru * ru);
    PairStream r(id, step, purpose, pkey);
    float g = 0.f;
    for (int t = 0; t < 128; ++t) {
        const uint2 w = r.next();
        const float a = 2.f * u01f(w.x) - 1.f;
        const float b = 2.f * u01f(w.y) - 1.f;
        const float s = a * a + b * b;
        if (s < 1.f && s > 0.f) {
            g = a * sqrtf(__fdividef(-2.f * logf(s), s));
            break;
        }
    }
    const float d = sqrtf(sig2) * g;
    const float rden = __fdividef(1.f, 1.f + d * d);
    const float sn = 2.f * d * rden, omc = 2.f * d * d * rden;
    float a = 0.f, b = 0.f, s2 = 0.f;
    int t;
    for (t = 0; t < 128; ++t) {
        const uint2 w = r.next();
        a = 2.f * u01f(w.x) - 1.f;
        b = 2.f * u01f(w.y) - 1.f;
        s2 = a * a + b * b;
        if (s2 < 1.f && s2 > 0.f) break;
    }
    float cp = 1.f, sp = 0.f;
    if (t < 128) {
        const float rs = __fdividef(1.f, s2);
        cp = (a * a - b * b) * rs;
        sp = 2.f * a * b * rs;
    }
    const float up2 = u[0] * u[0] + u[1] * u[1];
    float du[3];
    if (up2 > 0.f) {
        const float rup = rsqrtf(up2);
        const float up = up2 * rup;
        const float c1 = u[2] * sn * cp * rup, c2 = um * sn * sp * rup;
        du[0] = u[0] * c1 - u[1] * c2 - u[0] * omc;
        du[1] = u[1] * c1 + u[0] * c2 - u[1] * omc;
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
    void* vel[2];
    double w, vol, dt;            // weight, cell volume, step
    double cf[3];                 // e-e, i-i, e-i: q^4 lnL / (8 pi eps0^2 mu^2) (SI); mixed: times dt / (dx/dt)^3
    double fac[2][2];             // mu / m_a of a pair of species (a, b), mu = m_a m_b / (m_a + m_b)
    float fac32[2][2], cf32[3];   // the same in float for the mixed pass
    float wv32;                   // w / vol in float
    const uint32_t* step;
    uint2 pkey;
};

// the partner density of a group of n particles (FP64: the oracle's operations)
__device__ __forceinline__ double density(const CoulArgs& a, unsigned int n, double*)
{
    return ((double)n * a.w) / a.vol;
}
__device__ __forceinline__ float density(const CoulArgs& a, unsigned int n, float*)
{
    return (float)n * a.wv32;
}

// entries of the parameter tables by selects (an indexed read would copy the
// kernel parameter to local memory)
template <typename X>
__device__ __forceinline__ X pick(const X (&v)[2][2], int x, int y)
{
    return x == 0 ? (y == 0 ? v[0][0] : v[0][1]) : (y == 0 ? v[1][0] : v[1][1]);
}
template <typename X>
__device__ __forceinline__ X pick(const X (&v)[3], int k)
{
    return k == 0 ? v[0] : k == 1 ? v[1] : v[2];
}

// one collision of slot qa (species sa, the pair's first particle) with slot qb
// (species sb); kind 0 e-e, 1 i-i, 2 e-i.  Whole records are read and written
// back; their fourth word (the id) passes through.
__device__ __forceinline__ void collide(const CoulArgs& a, int sa, unsigned int qa, int sb, unsigned int qb,
                                        int kind, double dens, bool half, uint32_t step, uint32_t purpose, double*)
{
    double4* pa = reinterpret_cast<double4*>(sa == 0 ? a.vel[0] : a.vel[1]) + qa;
    double4* pb = reinterpret_cast<double4*>(sb == 0 ? a.vel[0] : a.vel[1]) + qb;
    double4 A = *pa, B = *pb;
    double va[3] = {A.x, A.y, A.z}, vb[3] = {B.x, B.y, B.z};
    const double dt = half ? 0.5 * a.dt : a.dt;
    coul_pair64(va, vb, pick(a.fac, sa, sb), pick(a.fac, sb, sa), pick(a.cf, kind), dens, dt, coul_id(A), step,
                purpose, a.pkey);
    A.x = va[0]; A.y = va[1]; A.z = va[2];
    B.x = vb[0]; B.y = vb[1]; B.z = vb[2];
    *pa = A;
    *pb = B;
}
__device__ __forceinline__ void collide(const CoulArgs& a, int sa, unsigned int qa, int sb, unsigned int qb,
                                        int kind, float dens, bool half, uint32_t step, uint32_t purpose, float*)
{
    float4* pa = reinterpret_cast<float4*>(sa == 0 ? a.vel[0] : a.vel[1]) + qa;
    float4* pb = reinterpret_cast<float4*>(sb == 0 ? a.vel[0] : a.vel[1]) + qb;
    float4 A = *pa, B = *pb;
    float va[3] = {A.x, A.y, A.z}, vb[3] = {B.x, B.y, B.z};
    coul_pair32(va, vb, pick(a.fac32, sa, sb), pick(a.fac32, sb, sa), pick(a.cf32, kind), dens, half ? 0.5f : 1.f,
                coul_id(A), step, purpose, a.pkey);
    A.x = va[0]; A.y = va[1]; A.z = va[2];
    B.x = vb[0]; B.y = vb[1]; B.z = vb[2];
    *pa = A;
    *pb = B;
}

struct CoulGroups {
    const unsigned int* end[2];    // per species: end slot of each cell's group
    const unsigned int* cell[2];   // cell of each grouped slot
    unsigned int cells;
};

// grouped particles of each species: the end of the last cell's group
__device__ __forceinline__ void group_totals(const CoulGroups& g, unsigned int& n0, unsigned int& n1)
{
    n0 = g.end[0][g.cells - 1];
    n1 = g.end[1][g.cells - 1];
}

__device__ __forceinline__ void group_of(const CoulGroups& g, int sp, unsigned int c, unsigned int& b0,
                                         unsigned int& b1)
{
    const unsigned int* e = sp == 0 ? g.end[0] : g.end[1];   // (a select: no indexed copy of the parameter)
    b0 = c == 0 ? 0u : e[c - 1];
    b1 = e[c];
}

// rank of each grouped particle's key among its cell's keys -> key order
__global__ void __launch_bounds__(256) k_coul_rank(const CoulGroups g, const unsigned long long* key_e,
                                                   const unsigned long long* key_i, const unsigned int* idx_e,
                                                   const unsigned int* idx_i, unsigned int* ord_e,
                                                   unsigned int* ord_i)
{
    unsigned int n0, n1;
    group_totals(g, n0, n1);
    const unsigned long long total = (unsigned long long)n0 + n1;
    for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < total;
         t += (unsigned long long)gridDim.x * blockDim.x) {
        const int sp = t < n0 ? 0 : 1;
        const unsigned int d = (unsigned int)(sp == 0 ? t : t - n0);
        const unsigned long long* key = sp == 0 ? key_e : key_i;
        unsigned int b0, b1;
        group_of(g, sp, (sp == 0 ? g.cell[0] : g.cell[1])[d], b0, b1);
        const unsigned long long k = key[d];
        unsigned int r = 0;
        for (unsigned int j = b0; j < b1; ++j) r += key[j] < k;     // keys are unique (they end with the id)
        (sp == 0 ? ord_e : ord_i)[b0 + r] = (sp == 0 ? idx_e : idx_i)[d];
    }
}

// Collision work is staged per warp: a pass over 32 grouped particles
// appends each item it finds (a like pair, a like triplet, or a particle of
// the smaller group of a cell with its e-Ar+ partners) to the warp's queue in
// shared memory, and 32 queued items at a time go to the 32 lanes.  Each lane
// makes one collision of its item and, when the item has more (the next
// collision of a triplet, the next partner of an e-Ar+ item), puts it back in
// the queue, so every lane of a round collides exactly once.  A particle is in
// one item only and its item is queued once at a time, so each particle meets
// its partners in order; items touch disjoint particles, so their order is free.
constexpr int kWarps = 8;   // warps of a 256-thread block
#ifndef PIC_COUL_MINB       // resident blocks per SM the collision kernels are built for
#ifdef PIC_COUL_MIXED
#define PIC_COUL_MINB 4
#else
#define PIC_COUL_MINB 2
#endif
#endif

struct WarpQueue {
    uint4* it;        // 64 entries in shared memory
    unsigned int n;   // queued items (warp-uniform); below 32 between rounds

    // append this lane's item (if any); all lanes call
    __device__ __forceinline__ void push(bool has, const uint4& v)
    {
        const unsigned int lane = threadIdx.x & 31u;
        const unsigned int m = __ballot_sync(0xffffffffu, has);
        if (has) it[n + __popc(m & ((1u << lane) - 1u))] = v;
        n += __popc(m);
        __syncwarp();
    }
    // rounds of 32 items while 32 are queued (while any is, when `all`); `step`
    // makes one collision and returns whether the item, updated in place,
    // has another; all lanes call
    template <typename F>
    __device__ __forceinline__ void drain(bool all, F&& step)
    {
        const unsigned int lane = threadIdx.x & 31u;
        while (n >= 32u || (all && n > 0u)) {
            const unsigned int take = n >= 32u ? 32u : n;
            n -= take;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (lane < take) v = it[n + lane];
            __syncwarp();
            const bool more = lane < take && step(v);
            push(more, v);
        }
    }
};

// the warps of the grid walk the grouped particles (both species, electrons
// first) 32 at a time
#define PIC_COUL_WARP_LOOP(total)                                                                          \
    for (unsigned long long base = (blockIdx.x * (unsigned long long)kWarps + (threadIdx.x >> 5)) * 32ull; \
         base < (total); base += gridDim.x * (unsigned long long)kWarps * 32ull)

// like pairs: in a group of n in key order, (0,1), (2,3), ... for even n; for
// odd n the triplet (0,1), (1,2), (2,0) at half the step, then (3,4), (5,6), ...
// An item is (group start, position of its first particle, n, species | stage
// << 1): stage 0 a pair, 1..3 the triplet's collisions in order.
template <typename T>
__global__ void __launch_bounds__(256, PIC_COUL_MINB) k_coul_like(const CoulArgs a, const CoulGroups g,
                                                                  const unsigned int* ord_e,
                                                                  const unsigned int* ord_i)
{
    __shared__ uint4 store[kWarps][64];
    const uint32_t step = *a.step - 1u;
    unsigned int n0, n1;
    group_totals(g, n0, n1);
    const unsigned long long total = (unsigned long long)n0 + n1;
    WarpQueue q{store[threadIdx.x >> 5], 0u};
    auto one = [&](uint4& it) -> bool {
        const int sp = (int)(it.w & 1u);
        const unsigned int stage = it.w >> 1;
        const unsigned int* L = (sp == 0 ? ord_e : ord_i) + it.x;
        const unsigned int ib = stage == 0u ? it.y + 1u : stage == 3u ? 0u : stage;
        const unsigned int ia = stage == 0u ? it.y : stage - 1u;
        collide(a, sp, L[ia], sp, L[ib], sp, density(a, it.z, (T*)nullptr), stage != 0u, step,
                sp == 0 ? kPurCoulEE : kPurCoulII, (T*)nullptr);
        it.w += 2u;
        return stage == 1u || stage == 2u;
    };
    PIC_COUL_WARP_LOOP(total)
    {
        const unsigned long long t = base + (threadIdx.x & 31u);
        bool has = false;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (t < total) {
            const int sp = t < n0 ? 0 : 1;
            const unsigned int d = (unsigned int)(sp == 0 ? t : t - n0);
            unsigned int b0, b1;
            group_of(g, sp, (sp == 0 ? g.cell[0] : g.cell[1])[d], b0, b1);
            const unsigned int n = b1 - b0, r = d - b0;
            if (n >= 2) {
                const bool trip = n % 2 == 1 && r == 0;
                has = trip || (n % 2 == 1 ? (r >= 3 && (r & 1) == 1) : (r & 1) == 0);
                v = make_uint4(b0, r, n, (unsigned int)sp | (trip ? 2u : 0u));
            }
        }
        q.push(has, v);
        q.drain(false, one);
    }
    q.drain(true, one);
}

// e-Ar+: every particle of the larger group A (electrons on a tie) meets
// B[k mod |B|] at the density of B; the item of B's position b takes
// k = b, b + |B|, ... in that order.  An item is (the ord index of A[k], B's
// slot, |B| | A's species << 31, collisions left).
template <typename T>
__global__ void __launch_bounds__(256, PIC_COUL_MINB) k_coul_unlike(const CoulArgs a, const CoulGroups g,
                                                                    const unsigned int* ord_e,
                                                                    const unsigned int* ord_i)
{
    __shared__ uint4 store[kWarps][64];
    const uint32_t step = *a.step - 1u;
    unsigned int n0, n1;
    group_totals(g, n0, n1);
    const unsigned long long total = (unsigned long long)n0 + n1;
    WarpQueue q{store[threadIdx.x >> 5], 0u};
    auto one = [&](uint4& it) -> bool {
        const int big = (int)(it.z >> 31);
        const unsigned int nb = it.z & 0x7fffffffu;
        const unsigned int qa = (big == 0 ? ord_e : ord_i)[it.x];
        collide(a, big, qa, 1 - big, it.y, 2, density(a, nb, (T*)nullptr), false, step, kPurCoulEI, (T*)nullptr);
        it.x += nb;
        it.w -= 1u;
        return it.w != 0u;
    };
    PIC_COUL_WARP_LOOP(total)
    {
        const unsigned long long t = base + (threadIdx.x & 31u);
        bool has = false;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (t < total) {
            const int sp = t < n0 ? 0 : 1;
            const unsigned int d = (unsigned int)(sp == 0 ? t : t - n0);
            const unsigned int c = (sp == 0 ? g.cell[0] : g.cell[1])[d];
            unsigned int e0, e1, i0, i1;
            group_of(g, 0, c, e0, e1);
            group_of(g, 1, c, i0, i1);
            const unsigned int ne = e1 - e0, ni = i1 - i0;
            const int big = ne >= ni ? 0 : 1;
            has = ne != 0 && ni != 0 && sp != big;   // the particles of the smaller group B
            if (has) {
                const unsigned int na = big == 0 ? ne : ni, nb = big == 0 ? ni : ne;
                const unsigned int b = d - (sp == 0 ? e0 : i0);
                const unsigned int qb = (sp == 0 ? ord_e : ord_i)[d];
                v = make_uint4((big == 0 ? e0 : i0) + b, qb, nb | ((unsigned int)big << 31),
                               (na - b + nb - 1u) / nb);
            }
        }
        q.push(has, v);
        q.drain(false, one);
    }
    q.drain(true, one);
}

#undef PIC_COUL_WARP_LOOP

}  // namespace

// One translation unit per precision: this file is compiled as is for the FP64
// pass (without fused multiply-add, bit-exact with the oracle) and through
// coulomb_mixed.cu with PIC_COUL_MIXED for the float pass (with FMA).
#ifdef PIC_COUL_MIXED
using CT = float;
using CT4 = float4;
#define PIC_COUL_LAUNCH launch_coulomb_mixed
#else
using CT = double;
using CT4 = double4;
#define PIC_COUL_LAUNCH launch_coulomb_fp64
#endif

void PIC_COUL_LAUNCH(pic_ctx* c)
{
    const bool mixed = c->prec == PIC_MIXED;
    const size_t nc = c->cells;
    CoulArgs a{};
    for (int sp = 0; sp < 2; ++sp) {
        cudaMemsetAsync(c->cs_end[sp], 0, sizeof(unsigned int) * nc, c->stream);
        const int grid = grid_for(c->cap[sp], 256, 152 * 8);
        k_coul_count<CT4><<<grid, 256, 0, c->stream>>>((const CT4*)c->pos[sp], c->d_nslot, sp, c->cs_end[sp],
                                                       c->nx, c->ny);
        scan_cells(c, c->cs_end[sp]);
        k_coul_scatter<CT4><<<grid, 256, 0, c->stream>>>((const CT4*)c->pos[sp], (const CT4*)c->vel[sp], c->d_nslot,
                                                         sp, c->cs_end[sp], c->cs_idx[sp], c->cs_key[sp],
                                                         c->cs_cell[sp], c->nx, c->ny, c->d_step, c->key);
        c->launches += 2;
        a.vel[sp] = c->vel[sp];
    }
    a.w = c->W;
    a.vol = c->dx * c->dx * c->dx;
    a.dt = c->dt;
    const double m[2] = {kME, kMAR};
    for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 2; ++y) {
            const double mu = (m[x] * m[y]) / (m[x] + m[y]);
            a.fac[x][y] = mu / m[x];
            a.fac32[x][y] = (float)a.fac[x][y];
        }
    a.wv32 = (float)(c->W / (c->dx * c->dx * c->dx));
    const double vs = c->dx / c->dt;
    for (int k = 0; k < 3; ++k) {
        const double ma = k == 1 ? kMAR : kME, mb = k == 0 ? kME : kMAR;
        const double mu = (ma * mb) / (ma + mb);
        const double cf = ((((kQE * kQE) * (kQE * kQE)) * c->coul_log) / (((8.0 * kPI) * (kEPS0 * kEPS0)) * (mu * mu)));
        a.cf[k] = mixed ? cf * c->dt / (vs * vs * vs) : cf;
        a.cf32[k] = (float)a.cf[k];
    }
    a.step = c->d_step;
    a.pkey = c->key;
    CoulGroups g{};
    for (int sp = 0; sp < 2; ++sp) {
        g.end[sp] = c->cs_end[sp];
        g.cell[sp] = c->cs_cell[sp];
    }
    g.cells = (unsigned int)nc;
    const int grid = grid_for(c->cap[0] + c->cap[1], 256, 152 * 16);
    // the collision kernels: one resident wave, so that each warp's queue runs
    // many full rounds before its last, partial ones
    const int gridc = std::min(grid, 152 * PIC_COUL_MINB);
    k_coul_rank<<<grid, 256, 0, c->stream>>>(g, c->cs_key[0], c->cs_key[1], c->cs_idx[0], c->cs_idx[1],
                                             c->cs_ord[0], c->cs_ord[1]);
    k_coul_like<CT><<<gridc, 256, 0, c->stream>>>(a, g, c->cs_ord[0], c->cs_ord[1]);
    k_coul_unlike<CT><<<gridc, 256, 0, c->stream>>>(a, g, c->cs_ord[0], c->cs_ord[1]);
    c->launches += 3;
}

#ifndef PIC_COUL_MIXED
void launch_coulomb(pic_ctx* c)
{
    if (c->prec == PIC_MIXED) launch_coulomb_mixed(c);
    else launch_coulomb_fp64(c);
}
#endif

}  // namespace pic

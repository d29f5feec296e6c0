// Mixed-precision particle cycle (Sec. III).  Same steps as the FP64 path
// (gather of -grad phi, Eqs. 1-2 leapfrog, MD subcycling with Eqs. 5-6 near
// grains, absorption, null-collision MCC of Table I, fixed-point CIC deposit)
// on a compact layout:
//   pos float4 {ox, oy, oz, cell}: in-cell offsets in [0,1) and the packed cell
//       (i | j << 10 | k << 20 as int bits; -1 = dead slot), so positions keep
//       ~6e-8 cell resolution anywhere in the box;
//   vel float4 {vx, vy, vz, id}: velocity in cells per step, particle id bits.
// The push works in cell units: v += (q/m) E dt^2/dx, offset += v, with the
// integer part carried into the cell.  Collisions convert to SI.
//
// One step runs three kernels per species:
//   k_push32  every particle outside the MD regions: gather, push, electrode
//             loss, the null-collision test, deposit.  The particles are
//             sorted by tile (8 x 8 x 8 cells); one thread block takes the slot
//             range of one tile as it stood at the last sort and sums its
//             deposits in a shared-memory window over the tile's nodes plus a
//             margin of `halo` cells (particles drift between sorts), flushed
//             with one global atomic per touched node.  Corners outside the
//             window, and the ionization products appended since the sort
//             (taken by extra blocks), go to global atomics.  Collision
//             candidates are appended to a list, particles that end in an MD
//             cell to the next step's MD list.
//   k_md32    the MD-region particles (listed during the previous step, so it
//             runs on a second stream alongside k_push32): Dt/40 substeps with
//             the PPPM correction, grain absorption, MCC, deposit.
//   k_mcc32   the collision candidates: process selection and kinematics.
// The ion push and its collisions run on a third stream beside the electron
// push: the species share only the charge array and the counters, both summed
// with atomics, so the overlap hides each launch's last partial wave.
#include <algorithm>
#include <climits>

#include "pic_internal.cuh"

namespace pic {
namespace {

#ifndef PIC_PUSH_PPT
#define PIC_PUSH_PPT 1
#endif
#ifndef PIC_PUSH_MINB
#define PIC_PUSH_MINB 5                           // resident blocks per SM the register budget is set for
#endif
#ifndef PIC_PUSH_TAIL
#define PIC_PUSH_TAIL 76                          // blocks for the particles appended since the last sort
#endif
constexpr int kPushThreads = 256;
constexpr int kPPT = PIC_PUSH_PPT;               // particles per thread per loop trip
constexpr int kTailBlocks = PIC_PUSH_TAIL;

struct P32 {
    int nx, ny, nz, nxy;
    int M, sp, flags;
    float kq, kqm, invM;         // (q/m) dt^2/dx, its per-substep value, 1/M
    float vs, inv_vs;            // dx/dt and its inverse (cells/step <-> m/s)
    float hm, pnull, nu_max, de, n_gas, sig_n, eps_exc, eps_ion, mr2, qk;
    int n_xs;
    const float* xs;
    uint2 key;
    const uint32_t* step;        // device step counter (Philox counter word 2)
    const int* gcell;
    const float* goff;           // 3 ng: grain centre offsets in its cell
    const float* gr2;            // ng: (radius/dx)^2
    const float* gq;             // ng: Q (C)
    const float* gtab;           // ng * 192: unit-charge node field (V/m per C)
    unsigned long long* gabs;
    const int* cell_ng;
    const int* cell_g;
    const float4* E;
    unsigned long long* rq;
    float4* pos;
    float4* vel;
    const unsigned long long* nslot;
    unsigned long long* cnt;
    int* err;
    ChildRec* child;
    unsigned long long child_cap;
    unsigned long long* nch;
    unsigned int* md_list;       // MD-region particles of this step (built during the previous one)
    unsigned int* md_n;
    unsigned int* md_next;       // ... and of the next step
    unsigned int* md_next_n;
    float4* md_res;              // MD results (pos, vel) per list entry, committed after the step's join
    unsigned int md_rescap;
    unsigned int* mcc_list;
    unsigned int* mcc_n;
    const unsigned int* tstart;  // first slot of each tile at the last sort (ntiles + 1)
    int tx, ty, tz, ntx, nty;    // tile edge (cells) and tiles per axis in x and y
    long long ntiles;
    int halo;                    // deposit window margin (cells)
    int wx, wy, wz;              // deposit window extent (nodes): tile + 1 + 2 halo per axis
};

enum Event : int { kEvNone = 0, kEvEEl, kEvEExc, kEvEIon, kEvIEl, kEvICx };

__device__ __forceinline__ void latch(int* err, int code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ int pack(int i, int j, int k) { return i | (j << 10) | (k << 20); }
__device__ __forceinline__ void unpack(int c, int& i, int& j, int& k)
{
    i = c & 1023;
    j = (c >> 10) & 1023;
    k = c >> 20;
}

__device__ __forceinline__ int qa(float o)
{
    const int a = __float2int_rn(o * (float)kWQ);
    return min(max(a, 0), kWQ);
}

// add `pred` lanes of the active threads of this warp to *ctr with one atomic
__device__ __forceinline__ void warp_count(unsigned long long* ctr, bool pred)
{
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, pred);
    if (m && (threadIdx.x & 31) == __ffs(act) - 1) atomicAdd(ctr, (unsigned long long)__popc(m));
}

// append q to a list with one atomic per warp
__device__ __forceinline__ void warp_append(unsigned int* list, unsigned int* n, unsigned int q, bool pred)
{
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, pred);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned int base = 0;
    if (lane == leader) base = atomicAdd(n, (unsigned int)__popc(m));
    base = __shfl_sync(act, base, leader);
    if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = q;
}

// Collision candidates of one block, staged in shared memory so that the
// global list counter takes one atomic per block instead of one per warp (the
// counter is shared by the whole grid and serialises in L2); entries beyond
// the stage go to the global list directly.
constexpr int kCandStage = 512;
struct CandStage {
    unsigned int n[2];
    unsigned int q[2][kCandStage];
};

__device__ __forceinline__ void stage_append(CandStage& st, int sp, unsigned int* list, unsigned int* n,
                                             unsigned int q, bool pred)
{
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, pred);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned int base = 0;
    if (lane == leader) base = atomicAdd(&st.n[sp], (unsigned int)__popc(m));
    base = __shfl_sync(act, base, leader);
    if (!pred) return;
    const unsigned int slot = base + (unsigned int)__popc(m & ((1u << lane) - 1u));
    if (slot < kCandStage) st.q[sp][slot] = q;
    else list[atomicAdd(n, 1u)] = q;
}

// the staged candidates of both species to the global lists (after a barrier)
__device__ __forceinline__ void stage_flush(CandStage& st, unsigned int* list_e, unsigned int* n_e,
                                            unsigned int* list_i, unsigned int* n_i)
{
    __shared__ unsigned int s_base[2];
    if (threadIdx.x < 2) {
        const unsigned int k = min(st.n[threadIdx.x], (unsigned int)kCandStage);
        s_base[threadIdx.x] = k ? atomicAdd(threadIdx.x == 0 ? n_e : n_i, k) : 0u;
    }
    __syncthreads();
    const unsigned int ke = min(st.n[0], (unsigned int)kCandStage), ki = min(st.n[1], (unsigned int)kCandStage);
    for (unsigned int t = threadIdx.x; t < ke; t += blockDim.x) list_e[s_base[0] + t] = st.q[0][t];
    for (unsigned int t = threadIdx.x; t < ki; t += blockDim.x) list_i[s_base[1] + t] = st.q[1][t];
}

// CIC gather of the node field with the fixed-point weights a/2^14 per axis
__device__ __forceinline__ void gather(const float4* __restrict__ E, int nx, int ny, int i, int j, int k,
                                       const int a[3], float out[3])
{
    const float s = 1.0f / (float)kWQ;
    const float wx0 = (float)(kWQ - a[0]) * s, wx1 = (float)a[0] * s;
    const float wy0 = (float)(kWQ - a[1]) * s, wy1 = (float)a[1] * s;
    const float wz0 = (float)(kWQ - a[2]) * s, wz1 = (float)a[2] * s;
    const int i1 = (i + 1 == nx) ? 0 : i + 1;
    const int j1 = (j + 1 == ny) ? 0 : j + 1;
    const int nxy = nx * ny;
    const int b0 = k * nxy, b1 = b0 + nxy;
    const int r00 = b0 + j * nx, r01 = b0 + j1 * nx, r10 = b1 + j * nx, r11 = b1 + j1 * nx;
    const float4 e000 = __ldg(E + r00 + i), e001 = __ldg(E + r00 + i1);
    const float4 e010 = __ldg(E + r01 + i), e011 = __ldg(E + r01 + i1);
    const float4 e100 = __ldg(E + r10 + i), e101 = __ldg(E + r10 + i1);
    const float4 e110 = __ldg(E + r11 + i), e111 = __ldg(E + r11 + i1);
    const float w00 = wy0 * wz0, w01 = wy1 * wz0, w10 = wy0 * wz1, w11 = wy1 * wz1;
    out[0] = w00 * (wx0 * e000.x + wx1 * e001.x) + w01 * (wx0 * e010.x + wx1 * e011.x) +
             w10 * (wx0 * e100.x + wx1 * e101.x) + w11 * (wx0 * e110.x + wx1 * e111.x);
    out[1] = w00 * (wx0 * e000.y + wx1 * e001.y) + w01 * (wx0 * e010.y + wx1 * e011.y) +
             w10 * (wx0 * e100.y + wx1 * e101.y) + w11 * (wx0 * e110.y + wx1 * e111.y);
    out[2] = w00 * (wx0 * e000.z + wx1 * e001.z) + w01 * (wx0 * e010.z + wx1 * e011.z) +
             w10 * (wx0 * e100.z + wx1 * e101.z) + w11 * (wx0 * e110.z + wx1 * e111.z);
}

// the 8 corner nodes and fixed-point weights of a particle
__device__ __forceinline__ void corners(int nx, int ny, int i, int j, int k, const int a[3], long long charge,
                                        int node[8], long long val[8])
{
    const int i1 = (i + 1 == nx) ? 0 : i + 1;
    const int j1 = (j + 1 == ny) ? 0 : j + 1;
    const int nxy = nx * ny;
    const int r0 = k * nxy + j * nx, r1 = k * nxy + j1 * nx;
    const int wx[2] = {kWQ - a[0], a[0]}, wy[2] = {kWQ - a[1], a[1]};
    const long long wz[2] = {charge * (kWQ - a[2]), charge * a[2]};
    const int ii[2] = {i, i1};
    const int rr[2] = {r0, r1};
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int di = 0; di < 2; ++di) {
                const int c = dz * 4 + dy * 2 + di;
                node[c] = rr[dy] + dz * nxy + ii[di];
                val[c] = (long long)(wx[di] * wy[dy]) * wz[dz];
            }
}

__device__ __forceinline__ void deposit_global(unsigned long long* rq, int nx, int ny, int i, int j, int k,
                                               const int a[3], long long charge)
{
    int node[8];
    long long val[8];
    corners(nx, ny, i, j, k, a, charge, node, val);
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (val[c] != 0) atomicAdd(rq + node[c], (unsigned long long)val[c]);
}

// carry whole cells out of the offsets; 0 alive, 1/2 lost at the bottom/top
// electrode, 3 invalid (non-finite or more than one box length in a step)
__device__ __forceinline__ int carry(int nx, int ny, int nz, int& i, int& j, int& k, float o[3])
{
    int c[3] = {i, j, k};
    const int n[3] = {nx, ny, nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!(fabsf(o[a]) < 1e6f)) return 3;
        const float fl = floorf(o[a]);
        o[a] -= fl;
        int cc = c[a] + (int)fl;
        if (o[a] >= 1.0f) { o[a] -= 1.0f; cc += 1; }
        if (a < 2) {
            if (cc < -n[a] || cc >= 2 * n[a]) return 3;
            if (cc < 0) cc += n[a];
            else if (cc >= n[a]) cc -= n[a];
        }
        c[a] = cc;
    }
    if (c[2] < 0) return 1;
    if (c[2] >= nz) return 2;
    i = c[0]; j = c[1]; k = c[2];
    return 0;
}

// separation from grain gi in cell units, minimum image in x and y
__device__ __forceinline__ void grain_sep(const P32& p, int gi, int i, int j, int k, const float o[3], float d[3])
{
    int di = i - p.gcell[3 * gi], dj = j - p.gcell[3 * gi + 1];
    const int dk = k - p.gcell[3 * gi + 2];
    if (di > p.nx / 2) di -= p.nx; else if (di < -p.nx / 2) di += p.nx;
    if (dj > p.ny / 2) dj -= p.ny; else if (dj < -p.ny / 2) dj += p.ny;
    d[0] = (float)di + (o[0] - p.goff[3 * gi]);
    d[1] = (float)dj + (o[1] - p.goff[3 * gi + 1]);
    d[2] = (float)dk + (o[2] - p.goff[3 * gi + 2]);
}

__device__ __forceinline__ float xs_at(const float* tab, int n, float de, float eps)
{
    const float t = eps / de;
    if (t >= (float)(n - 1)) return tab[n - 1];
    const int i = (int)t;
    const float fr = t - (float)i;
    return tab[i] + fr * (tab[i + 1] - tab[i]);
}

__device__ __forceinline__ void pairf(RStream& r, float& a, float& b)
{
    a = 2.0f * u01f(r.next()) - 1.0f;
    b = 2.0f * u01f(r.next()) - 1.0f;
}

__device__ void isof(RStream& r, float o[3])
{
    for (int t = 0; t < 128; ++t) {
        float a, b;
        pairf(r, a, b);
        const float s = a * a + b * b;
        if (s < 1.0f) {
            const float q = 2.0f * sqrtf(1.0f - s);
            o[0] = a * q; o[1] = b * q; o[2] = 1.0f - 2.0f * s;
            return;
        }
    }
    o[0] = 0.f; o[1] = 0.f; o[2] = 1.f;
}

__device__ void gauss3f(RStream& r, float o[3])
{
    int got = 0;
    for (int t = 0; t < 256 && got < 3; ++t) {
        float a, b;
        pairf(r, a, b);
        const float s = a * a + b * b;
        if (s < 1.0f && s > 0.0f) {
            const float f = sqrtf(-2.0f * logf(s) / s);
            o[got++] = a * f;
            if (got < 3) o[got++] = b * f;
        }
    }
    while (got < 3) o[got++] = 0.f;
}

// process selection and kinematics of a collision candidate (Table I), in SI
// single precision; u = the candidate's Philox draw (u.y picks the process)
__device__ int collide(const P32& p, uint32_t step, uint4 u, int cell, const float o[3], float vc[3], uint32_t id)
{
    float v[3] = {vc[0] * p.vs, vc[1] * p.vs, vc[2] * p.vs};
    const int nx = p.n_xs;
    if (p.sp == 0) {
        const float v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        const float eps = v2 * p.hm;
        const float vm = sqrtf(v2);
        const float nu_el = p.n_gas * xs_at(p.xs, nx, p.de, eps) * vm;
        const float nu_ex = p.n_gas * xs_at(p.xs + nx, nx, p.de, eps) * vm;
        const float nu_io = p.n_gas * xs_at(p.xs + 2 * nx, nx, p.de, eps) * vm;
        const float R = u01f(u.y) * p.nu_max;
        RStream rd(id, step, kPurDir, p.key);
        float dir[3];
        if (R < nu_el) {
            isof(rd, dir);
            const float cosx = (dir[0] * v[0] + dir[1] * v[1] + dir[2] * v[2]) / vm;
            const float vn = vm * sqrtf(1.0f - p.mr2 * (1.0f - cosx));
            for (int a = 0; a < 3; ++a) vc[a] = vn * dir[a] * p.inv_vs;
            return kEvEEl;
        }
        if (R < nu_el + nu_ex) {
            const float e2 = fmaxf(eps - p.eps_exc, 0.f);
            isof(rd, dir);
            const float vn = sqrtf(e2 / p.hm);
            for (int a = 0; a < 3; ++a) vc[a] = vn * dir[a] * p.inv_vs;
            return kEvEExc;
        }
        if (R < nu_el + nu_ex + nu_io) {
            const float e2 = fmaxf(eps - p.eps_ion, 0.f);
            const float vn = sqrtf(0.5f * e2 / p.hm);
            isof(rd, dir);
            float d2[3], gn[3];
            RStream rc(id, step, kPurChildDir, p.key);
            isof(rc, d2);
            RStream rn(id, step, kPurChildNeutral, p.key);
            gauss3f(rn, gn);
            ChildRec cr;
            cr.parent = id;
            cr.cell = cell;
            for (int a = 0; a < 3; ++a) {
                vc[a] = vn * dir[a] * p.inv_vs;
                cr.x[a] = o[a];
                cr.ve[a] = vn * d2[a] * p.inv_vs;
                cr.vi[a] = p.sig_n * gn[a] * p.inv_vs;
            }
            const unsigned long long slot = atomicAdd(p.nch, 1ull);
            if (slot < p.child_cap) p.child[slot] = cr;
            else latch(p.err, kErrCapacity);
            return kEvEIon;
        }
        return kEvNone;
    }
    float gn[3];
    RStream rn(id, step, kPurNeutral, p.key);
    gauss3f(rn, gn);
    const float vn[3] = {p.sig_n * gn[0], p.sig_n * gn[1], p.sig_n * gn[2]};
    const float gv[3] = {v[0] - vn[0], v[1] - vn[1], v[2] - vn[2]};
    const float g2 = gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2];
    const float eps = g2 * p.hm;
    const float gm = sqrtf(g2);
    const float nu_el = p.n_gas * xs_at(p.xs + 3 * nx, nx, p.de, eps) * gm;
    const float nu_cx = p.n_gas * xs_at(p.xs + 4 * nx, nx, p.de, eps) * gm;
    const float R = u01f(u.y) * p.nu_max;
    if (R < nu_el) {
        float dir[3];
        RStream rd(id, step, kPurDir, p.key);
        isof(rd, dir);
        for (int a = 0; a < 3; ++a) vc[a] = ((v[a] + vn[a]) * 0.5f + 0.5f * gm * dir[a]) * p.inv_vs;
        return kEvIEl;
    }
    if (R < nu_el + nu_cx) {
        for (int a = 0; a < 3; ++a) vc[a] = vn[a] * p.inv_vs;
        return kEvICx;
    }
    return kEvNone;
}

__device__ __forceinline__ void count_event(const P32& p, int ev)
{
    const int slot = ev == kEvEEl ? PIC_C_E_EL : ev == kEvEExc ? PIC_C_E_EXC : ev == kEvEIon ? PIC_C_E_ION
                   : ev == kEvIEl ? PIC_C_I_EL : PIC_C_I_CX;
    if (ev != kEvNone) atomicAdd(p.cnt + slot, 1ull);
}

// Window-relative coordinate of node index `n` along a periodic axis of
// length `len`, for a window starting at `o` (o may be negative): in [0, len).
__device__ __forceinline__ int wrel(int n, int o, int len)
{
    int d = n - o;
    if (d < 0) d += len;
    else if (d >= len) d -= len;
    return d;
}

// Exact 64-bit sums in the shared window from 32-bit shared atomics (a native
// 32-bit add is far cheaper than a 64-bit one): the low words at win32[s], the
// high words at win32[wn + s]; the carry out of the low word is detected from
// the value the low add returned.  Sums are modulo 2^64, so two's-complement
// (negative) contributions add correctly.
__device__ __forceinline__ void win_add(unsigned int* win32, int wn, int s, unsigned long long v)
{
    const unsigned int lo = (unsigned int)v, hi = (unsigned int)(v >> 32);
    const unsigned int old = atomicAdd(win32 + s, lo);
    atomicAdd(win32 + wn + s, hi + (old + lo < old ? 1u : 0u));
}

// The particles of one species in slots [first, end) with block-uniform trips
// of kPPT x kPushThreads (every lane of a warp takes every trip: warp votes
// below).  Deposits go to the block's window (signed sums) when all 8 corners
// fall inside it, else to global atomics.
__device__ __forceinline__ void push_range(const P32& p, unsigned long long first, unsigned long long end,
                                           unsigned long long stride, bool tiled, int ox, int oy, int oz,
                                           unsigned int* win, CandStage& cst, uint32_t step,
                                           unsigned int& live)
{
    const int wn = p.wx * p.wy * p.wz;
    const bool frozen = (p.sp == 1) && (p.flags & PIC_F_IONS_FROZEN);
    const bool no_mcc = p.flags & PIC_F_NO_MCC;
    const long long charge = p.sp == 0 ? -1 : 1;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int wx = p.wx, wy = p.wy, wz = p.wz, wxy = wx * wy;
    for (unsigned long long q0 = first; q0 < end; q0 += stride) {
        int dcell[kPPT];
        int da[kPPT][3];
        float4 Pr[kPPT], Vr[kPPT];
        // both records of every particle of the trip in flight at once; they stream
        // through once (evict-first), so the charge and field arrays keep L2
#pragma unroll
        for (int u = 0; u < kPPT; ++u) {
            const unsigned long long q = q0 + (unsigned long long)u * kPushThreads + threadIdx.x;
            Pr[u] = q < end ? __ldcs(p.pos + q) : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
            Vr[u] = q < end ? __ldcs(p.vel + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kPPT; ++u) {
            dcell[u] = -1;
            const unsigned long long q = q0 + (unsigned long long)u * kPushThreads + threadIdx.x;
            int lost = 0;
            bool md = false, cand = false;
            const float4 Pu = Pr[u];
            int cell = __float_as_int(Pu.w);
            if (cell >= 0) {
                ++live;
                int i, j, k;
                unpack(cell, i, j, k);
                float o[3] = {Pu.x, Pu.y, Pu.z};
                if (frozen) {
                    dcell[u] = cell;
                    da[u][0] = qa(o[0]); da[u][1] = qa(o[1]); da[u][2] = qa(o[2]);
                } else if (p.cell_ng[(k * ny + j) * nx + i] != 0) {
                    // in an MD region: on this step's MD list, advanced by k_md32
                } else {
                    const float4 Vu = Vr[u];
                    float v[3] = {Vu.x, Vu.y, Vu.z};
                    int a[3] = {qa(o[0]), qa(o[1]), qa(o[2])};
                    float E[3];
                    gather(p.E, nx, ny, i, j, k, a, E);
                    v[0] += E[0] * p.kq; v[1] += E[1] * p.kq; v[2] += E[2] * p.kq;
                    o[0] += v[0]; o[1] += v[1]; o[2] += v[2];
                    lost = carry(nx, ny, nz, i, j, k, o);
                    if (lost) {
                        p.pos[q].w = __int_as_float(-1);
                    } else {
                        if (!no_mcc) {
                            const uint4 r = philox4x32_10(make_uint4(__float_as_uint(Vu.w), step, kPurMCC, 0u),
                                                          p.key);
                            cand = u01f(r.x) < p.pnull;
                        }
                        cell = pack(i, j, k);
                        __stcs(p.pos + q, make_float4(o[0], o[1], o[2], __int_as_float(cell)));
                        __stcs(p.vel + q, make_float4(v[0], v[1], v[2], Vu.w));
                        dcell[u] = cell;
                        da[u][0] = qa(o[0]); da[u][1] = qa(o[1]); da[u][2] = qa(o[2]);
                        md = p.cell_ng[(k * ny + j) * nx + i] != 0;    // in an MD region next step
                    }
                }
            }
            if (__any_sync(0xffffffffu, md || cand || lost)) {
                warp_append(p.md_next, p.md_next_n, (unsigned int)q, md);
                stage_append(cst, p.sp, p.mcc_list, p.mcc_n, (unsigned int)q, cand);
                if (__any_sync(0xffffffffu, lost != 0)) {
                    warp_count(p.cnt + (p.sp == 0 ? PIC_C_LOST_BOT_E : PIC_C_LOST_BOT_I), lost == 1);
                    warp_count(p.cnt + (p.sp == 0 ? PIC_C_LOST_TOP_E : PIC_C_LOST_TOP_I), lost == 2);
                    warp_count(p.cnt + PIC_C_ERR, lost == 3);
                    if (lost == 3) latch(p.err, kErrNonFinite);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kPPT; ++u) {
            if (dcell[u] < 0) continue;
            int i, j, k;
            unpack(dcell[u], i, j, k);
            const int di = wrel(i, ox, nx), dj = wrel(j, oy, ny), dk = k - oz;
            if (tiled && di + 1 < wx && dj + 1 < wy && dk >= 0 && dk + 1 < wz) {
                const int s0 = (dk * wy + dj) * wx + di;
                // corner weight wx (< 2^15) x wy wz (< 2^29): one 32 x 32 -> 64-bit product;
                // electrons add the two's complement (the window holds signed sums)
                const unsigned int wxs[2] = {(unsigned int)(kWQ - da[u][0]), (unsigned int)da[u][0]};
                const unsigned int wyz[4] = {(unsigned int)((kWQ - da[u][1]) * (kWQ - da[u][2])),
                                             (unsigned int)(da[u][1] * (kWQ - da[u][2])),
                                             (unsigned int)((kWQ - da[u][1]) * da[u][2]),
                                             (unsigned int)(da[u][1] * da[u][2])};
                const int off[4] = {0, wx, wxy, wxy + wx};
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const unsigned long long v = (unsigned long long)wxs[c & 1] * wyz[c >> 1];
                    win_add(win, wn, s0 + off[c >> 1] + (c & 1), charge < 0 ? 0ull - v : v);
                }
            } else {
                deposit_global(p.rq, nx, ny, i, j, k, da[u], charge);
            }
        }
    }
}

// Blocks [0, ntiles): the electrons, then the ions, of one tile (their slot
// ranges at the last sort), deposits of both summed in one shared window of
// wx x wy x wz nodes from the tile's lower corner minus `halo` cells, flushed
// once.  Blocks [ntiles, grid): the ionization products appended since the
// sort, deposited with global atomics.
__global__ void __launch_bounds__(kPushThreads, PIC_PUSH_MINB) k_push32(const P32 pe, const P32 pi)
{
    extern __shared__ unsigned int win[];          // low words [0, wn), high words [wn, 2 wn)
    __shared__ CandStage cst;
    __shared__ unsigned int s_live;
    const uint32_t step = *pe.step;
    const int nx = pe.nx, ny = pe.ny;
    const int wx = pe.wx, wy = pe.wy, wz = pe.wz, wxy = wx * wy, wn = wxy * wz;
    const long long b = blockIdx.x;
    const bool tiled = b < pe.ntiles;
    unsigned int live = 0;
    if (tiled) {
        const unsigned long long e0 = pe.tstart[b], e1 = pe.tstart[b + 1];
        const unsigned long long i0 = pi.tstart[b], i1 = pi.tstart[b + 1];
        if (e0 == e1 && i0 == i1) return;                       // the whole block leaves together
        const int ti = (int)(b % pe.ntx), tj = (int)((b / pe.ntx) % pe.nty),
                  tk = (int)(b / ((long long)pe.ntx * pe.nty));
        const int ox = ti * pe.tx - pe.halo, oy = tj * pe.ty - pe.halo, oz = tk * pe.tz - pe.halo;
        for (int t = threadIdx.x; t < 2 * wn; t += blockDim.x) win[t] = 0u;
        if (threadIdx.x < 2) cst.n[threadIdx.x] = 0u;
        if (threadIdx.x == 0) s_live = 0u;
        __syncthreads();
        const unsigned long long stride = (unsigned long long)kPushThreads * kPPT;
        push_range(pe, e0, e1, stride, true, ox, oy, oz, win, cst, step, live);
        push_range(pi, i0, i1, stride, true, ox, oy, oz, win, cst, step, live);
        __syncthreads();
        // flush: each pass takes blockDim / wx whole window rows, one thread per node
        const int rows_per_pass = blockDim.x / wx;
        const int dxi = threadIdx.x - (threadIdx.x / wx) * wx;
        const int I = ((ox + dxi) % nx + nx) % nx;
        if ((int)threadIdx.x < rows_per_pass * wx)
            for (int row = threadIdx.x / wx; row < wy * wz; row += rows_per_pass) {
                const int t = row * wx + dxi;
                const unsigned long long v = ((unsigned long long)win[wn + t] << 32) | win[t];
                if (v == 0ull) continue;
                const int dz = row / wy, dy = row - dz * wy;
                const int J = ((oy + dy) % ny + ny) % ny;
                atomicAdd(pe.rq + ((size_t)(oz + dz) * ny + J) * nx + I, v);
            }
    } else {
        if (threadIdx.x < 2) cst.n[threadIdx.x] = 0u;
        if (threadIdx.x == 0) s_live = 0u;
        __syncthreads();
        const unsigned long long tb = (unsigned long long)(b - pe.ntiles) * kPushThreads * kPPT;
        const unsigned long long stride = (unsigned long long)(gridDim.x - pe.ntiles) * kPushThreads * kPPT;
        push_range(pe, pe.tstart[pe.ntiles] + tb, pe.nslot[0], stride, false, 0, 0, 0, win, cst, step, live);
        push_range(pi, pi.tstart[pi.ntiles] + tb, pi.nslot[1], stride, false, 0, 0, 0, win, cst, step, live);
        __syncthreads();
    }
    // one global atomic per block for the candidates of each species and the live count
    stage_flush(cst, pe.mcc_list, pe.mcc_n, pi.mcc_list, pi.mcc_n);
    live = __reduce_add_sync(0xffffffffu, live);
    if ((threadIdx.x & 31) == 0 && live) atomicAdd(&s_live, live);
    __syncthreads();
    if (threadIdx.x == 0 && s_live) atomicAdd(pe.cnt + PIC_C_PUSHED, (unsigned long long)s_live);
}

// Field data of one cell for the MD substeps: the 8 corner values of
// E_PIC - sum_g Q_g g_g (Eq. 5, mesh part) and the cell's near grains, so a
// substep that stays in its cell touches no memory.
struct MdCell {
    float ec[8][3];
    int ng;
    int gi[kMaxG];
};

__device__ void md_load(const P32& p, int i, int j, int k, MdCell& m)
{
    const int i1 = (i + 1 == p.nx) ? 0 : i + 1;
    const int j1 = (j + 1 == p.ny) ? 0 : j + 1;
    const int ii[2] = {i, i1}, jj[2] = {j, j1};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float4 e = __ldg(p.E + ((k + (c >> 2)) * p.ny + jj[(c >> 1) & 1]) * p.nx + ii[c & 1]);
        m.ec[c][0] = e.x; m.ec[c][1] = e.y; m.ec[c][2] = e.z;
    }
    const int cell = (k * p.ny + j) * p.nx + i;
    m.ng = p.cell_ng[cell];
    for (int t = 0; t < m.ng; ++t) {
        const int gi = p.cell_g[cell * kMaxG + t];
        m.gi[t] = gi;
        const float Q = p.gq[gi];
        const int gc0 = p.gcell[3 * gi], gc1 = p.gcell[3 * gi + 1], gc2 = p.gcell[3 * gi + 2];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int li = ((i + (c & 1) - gc0 + 1) % p.nx + p.nx) % p.nx;
            const int lj = ((j + ((c >> 1) & 1) - gc1 + 1) % p.ny + p.ny) % p.ny;
            const int lk = k + (c >> 2) - gc2 + 1;
            const float* tv = p.gtab + ((size_t)gi * 64 + (lk * 4 + lj) * 4 + li) * 3;
            m.ec[c][0] -= Q * tv[0];
            m.ec[c][1] -= Q * tv[1];
            m.ec[c][2] -= Q * tv[2];
        }
    }
}

// MD-region particles: md_sub substeps of dt/md_sub with the PPPM correction,
// absorption after each substep, then MCC and the deposit (Sec. III).  Runs
// beside k_push32, so the new states go to md_res and reach pos/vel only in
// k_md_commit, after both have finished (k_push32 reads these slots' cells).
__global__ void __launch_bounds__(64) k_md32(const P32 p)
{
    if (p.sp == 1 && (p.flags & PIC_F_IONS_FROZEN)) return;
    const unsigned int n = *p.md_n;
    const uint32_t step = *p.step;
    const long long charge = p.sp == 0 ? -1 : 1;
    const float s = 1.0f / (float)kWQ;
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const unsigned int q = p.md_list[t];
        const float4 P = p.pos[q];
        const float4 V = p.vel[q];
        if (t >= p.md_rescap) {            // no room for the result: leave the particle, report
            latch(p.err, kErrCapacity);
            continue;
        }
        int i, j, k;
        unpack(__float_as_int(P.w), i, j, k);
        float o[3] = {P.x, P.y, P.z};
        float v[3] = {V.x, V.y, V.z};
        int fate = 0, grain = -1;
        MdCell mc;
        md_load(p, i, j, k, mc);
        for (int m = 0; m < p.M; ++m) {
            const int a0 = qa(o[0]), a1 = qa(o[1]), a2 = qa(o[2]);
            const float wx[2] = {(float)(kWQ - a0) * s, (float)a0 * s};
            const float wy[2] = {(float)(kWQ - a1) * s, (float)a1 * s};
            const float wz[2] = {(float)(kWQ - a2) * s, (float)a2 * s};
            float E[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float w = wx[c & 1] * wy[(c >> 1) & 1] * wz[c >> 2];
                E[0] += w * mc.ec[c][0];
                E[1] += w * mc.ec[c][1];
                E[2] += w * mc.ec[c][2];
            }
            for (int g = 0; g < mc.ng; ++g) {      // Eq. 6: Coulomb field of the near grains
                float d[3];
                grain_sep(p, mc.gi[g], i, j, k, o, d);
                const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                const float coef = r2 > 0.f ? (p.gq[mc.gi[g]] * p.qk) / (r2 * sqrtf(r2)) : 0.f;
                E[0] += coef * d[0]; E[1] += coef * d[1]; E[2] += coef * d[2];
            }
            v[0] += E[0] * p.kqm; v[1] += E[1] * p.kqm; v[2] += E[2] * p.kqm;
            o[0] += v[0] * p.invM; o[1] += v[1] * p.invM; o[2] += v[2] * p.invM;
            const int pi = i, pj = j, pk = k;
            fate = carry(p.nx, p.ny, p.nz, i, j, k, o);
            if (fate) break;
            if (i != pi || j != pj || k != pk) md_load(p, i, j, k, mc);
            for (int g = 0; g < mc.ng && grain < 0; ++g) {
                float d[3];
                grain_sep(p, mc.gi[g], i, j, k, o, d);
                if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] <= p.gr2[mc.gi[g]]) grain = mc.gi[g];
            }
            if (grain >= 0) break;
        }
        if (fate != 0 || grain >= 0) {
            p.md_res[2 * t] = make_float4(P.x, P.y, P.z, __int_as_float(-1));
            p.md_res[2 * t + 1] = V;
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
        const int cell = pack(i, j, k);
        const uint32_t id = __float_as_uint(V.w);
        if (!(p.flags & PIC_F_NO_MCC)) {
            const uint4 r = philox4x32_10(make_uint4(id, step, kPurMCC, 0u), p.key);
            if (u01f(r.x) < p.pnull) count_event(p, collide(p, step, r, cell, o, v, id));
        }
        p.md_res[2 * t] = make_float4(o[0], o[1], o[2], __int_as_float(cell));
        p.md_res[2 * t + 1] = make_float4(v[0], v[1], v[2], V.w);
        const int a[3] = {qa(o[0]), qa(o[1]), qa(o[2])};
        deposit_global(p.rq, p.nx, p.ny, i, j, k, a, charge);
        if (p.cell_ng[(k * p.ny + j) * p.nx + i] != 0) p.md_next[atomicAdd(p.md_next_n, 1u)] = q;
    }
}

// write the MD results back once k_push32 and k_md32 have both finished
__global__ void k_md_commit(float4* pos_e, float4* vel_e, const unsigned int* list_e, const float4* res_e,
                            float4* pos_i, float4* vel_i, const unsigned int* list_i, const float4* res_i,
                            const unsigned int* lists, unsigned int rescap, int frozen_ions)
{
    const unsigned int ne = min(lists[0], rescap), ni = frozen_ions ? 0u : min(lists[2], rescap);
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < ne; t += gridDim.x * blockDim.x) {
        pos_e[list_e[t]] = res_e[2 * t];
        vel_e[list_e[t]] = res_e[2 * t + 1];
    }
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < ni; t += gridDim.x * blockDim.x) {
        pos_i[list_i[t]] = res_i[2 * t];
        vel_i[list_i[t]] = res_i[2 * t + 1];
    }
}

// start of a step: this step's MD lists are the ones built during the last step
__global__ void k_md_rotate(unsigned int* md_e, unsigned int* next_e, unsigned int* md_i, unsigned int* next_i,
                            unsigned int* lists)
{
    const unsigned int ne = lists[4], ni = lists[5];
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < ne; t += gridDim.x * blockDim.x)
        md_e[t] = next_e[t];
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < ni; t += gridDim.x * blockDim.x)
        md_i[t] = next_i[t];
}

__global__ void k_md_counts(unsigned int* lists)
{
    lists[0] = lists[4];     // md_n e
    lists[2] = lists[5];     // md_n i
    lists[1] = 0u;           // mcc_n e
    lists[3] = 0u;           // mcc_n i
    lists[4] = 0u;
    lists[5] = 0u;
}

// collision candidates found by k_push32 (their positions are final)
__global__ void __launch_bounds__(256) k_mcc32(const P32 p)
{
    const unsigned int n = *p.mcc_n;
    const uint32_t step = *p.step;
    for (unsigned int t0 = blockIdx.x * blockDim.x; t0 < n; t0 += gridDim.x * blockDim.x) {
        const unsigned int t = t0 + threadIdx.x;
        int ev = kEvNone;
        if (t < n) {
            const unsigned int q = p.mcc_list[t];
            const float4 P = p.pos[q];
            const float4 V = p.vel[q];
            const uint32_t id = __float_as_uint(V.w);
            const uint4 r = philox4x32_10(make_uint4(id, step, kPurMCC, 0u), p.key);
            float v[3] = {V.x, V.y, V.z};
            const float o[3] = {P.x, P.y, P.z};
            ev = collide(p, step, r, __float_as_int(P.w), o, v, id);
            if (ev != kEvNone) p.vel[q] = make_float4(v[0], v[1], v[2], V.w);
        }
        if (p.sp == 0) {
            warp_count(p.cnt + PIC_C_E_EL, ev == kEvEEl);
            warp_count(p.cnt + PIC_C_E_EXC, ev == kEvEExc);
            warp_count(p.cnt + PIC_C_E_ION, ev == kEvEIon);
        } else {
            warp_count(p.cnt + PIC_C_I_EL, ev == kEvIEl);
            warp_count(p.cnt + PIC_C_I_CX, ev == kEvICx);
        }
    }
}

__global__ void k_deposit32(int nx, int ny, const float4* pos, const unsigned long long* nslot, int sp,
                            unsigned long long* rq)
{
    const unsigned long long n = nslot[sp];
    const long long charge = sp == 0 ? -1 : 1;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const float4 P = pos[q];
        const int cell = __float_as_int(P.w);
        if (cell < 0) continue;
        int i, j, k;
        unpack(cell, i, j, k);
        const int a[3] = {qa(P.x), qa(P.y), qa(P.z)};
        deposit_global(rq, nx, ny, i, j, k, a, charge);
    }
}

// E = -grad phi on every node from the double-float potential: central
// differences in x, y and between the electrode planes, second-order one-sided
// differences on the planes.  Each difference of neighbouring values is taken
// part by part, (hi_a - hi_b) + (lo_a - lo_b), and rounded once to float.
__global__ void k_efield32(int nx, int ny, int nz, float inv_2dx, const float2* __restrict__ phi,
                           float4* __restrict__ E)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const int P = nx * ny;
    const int n = k * P + j * nx + i;
    const int row = n - i;
    const float2 xm = phi[row + (i == 0 ? nx - 1 : i - 1)], xp = phi[row + (i + 1 == nx ? 0 : i + 1)];
    const float2 ym = phi[k * P + (j == 0 ? ny - 1 : j - 1) * nx + i], yp = phi[k * P + (j + 1 == ny ? 0 : j + 1) * nx + i];
    const float ex = ((xm.x - xp.x) + (xm.y - xp.y)) * inv_2dx;
    const float ey = ((ym.x - yp.x) + (ym.y - yp.y)) * inv_2dx;
    float ez;
    if (k == 0 || k == nz) {
        // 3 phi_0 - 4 phi_1 + phi_2 = 3 (phi_0 - phi_1) - (phi_1 - phi_2), planes counted inwards
        const int s = k == 0 ? P : -P;
        const float2 a = phi[n], b = phi[n + s], c = phi[n + 2 * s];
        const float d01 = (a.x - b.x) + (a.y - b.y), d12 = (b.x - c.x) + (b.y - c.y);
        ez = (3.f * d01 - d12) * inv_2dx;
        if (k == nz) ez = -ez;
    } else {
        const float2 zm = phi[n - P], zp = phi[n + P];
        ez = ((zm.x - zp.x) + (zm.y - zp.y)) * inv_2dx;
    }
    E[n] = make_float4(ex, ey, ez, 0.f);
}

__global__ void k_children32(int nx, int ny, ChildRec* rec, const unsigned long long* nch,
                             unsigned long long child_cap, const unsigned long long* nslot,
                             const unsigned int* next_id, float4* pos_e, float4* vel_e, float4* pos_i,
                             float4* vel_i, long long cap_e, long long cap_i, unsigned long long* rq, int* err,
                             const int* cell_ng, unsigned int* next_e, unsigned int* next_i, unsigned int* lists)
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
        const float o[3] = {(float)cr.x[0], (float)cr.x[1], (float)cr.x[2]};
        const float cb = __int_as_float(cr.cell);
        pos_e[se] = make_float4(o[0], o[1], o[2], cb);
        vel_e[se] = make_float4((float)cr.ve[0], (float)cr.ve[1], (float)cr.ve[2],
                                __uint_as_float(nid + (unsigned)(2 * rank)));
        pos_i[si] = make_float4(o[0], o[1], o[2], cb);
        vel_i[si] = make_float4((float)cr.vi[0], (float)cr.vi[1], (float)cr.vi[2],
                                __uint_as_float(nid + (unsigned)(2 * rank + 1)));
        int i, j, k;
        unpack(cr.cell, i, j, k);
        const int a[3] = {qa(o[0]), qa(o[1]), qa(o[2])};
        deposit_global(rq, nx, ny, i, j, k, a, -1);
        deposit_global(rq, nx, ny, i, j, k, a, 1);
        if (next_e && cell_ng[(k * ny + j) * nx + i] != 0) {
            next_e[atomicAdd(lists + 4, 1u)] = (unsigned int)se;
            next_i[atomicAdd(lists + 5, 1u)] = (unsigned int)si;
        }
    }
}

__global__ void k_children_finish32(unsigned long long* nch, unsigned long long child_cap,
                                    unsigned long long* nslot, unsigned int* next_id, long long cap_e, long long cap_i,
                                    uint32_t* step)
{
    *step += 1u;   // the step is complete on the particle side
    const unsigned long long n = min(*nch, child_cap);
    nslot[0] = min(nslot[0] + n, (unsigned long long)cap_e);
    nslot[1] = min(nslot[1] + n, (unsigned long long)cap_i);
    *next_id += (unsigned int)(2 * n);
    *nch = 0;
}

// Node moments of one sample, in float: FP64 arithmetic issues at a small
// fraction of the FP32 rate on this GPU, so the CIC weights, weight x v and
// weight x |v|^2 are formed and summed in float (a node takes tens of adds per
// sample: about 1e-7 relative rounding), the first four as one float4
// reduction; k_mom_fold then adds them once per node to the FP64 window of the
// sample's phase bin.
__global__ void k_moments32(int nx, int ny, float vs, const float4* pos, const float4* vel,
                            const unsigned long long* nslot, int sp, float4* m4, float* mk)
{
    const unsigned long long n = nslot[sp];
    const float s = 1.0f / (float)kWQ;
    const int nxy = nx * ny;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        const float4 P = pos[q];
        const int cell = __float_as_int(P.w);
        if (cell < 0) continue;
        const float4 V = vel[q];
        int i, j, k;
        unpack(cell, i, j, k);
        const int ax = qa(P.x), ay = qa(P.y), az = qa(P.z);
        const float wx[2] = {(float)(kWQ - ax) * s, (float)ax * s};
        const float wy[2] = {(float)(kWQ - ay) * s, (float)ay * s};
        const float wz[2] = {(float)(kWQ - az) * s, (float)az * s};
        const int ii[2] = {i, (i + 1 == nx) ? 0 : i + 1};
        const int rr[2] = {j * nx, ((j + 1 == ny) ? 0 : j + 1) * nx};
        const float vx = V.x * vs, vy = V.y * vs, vz = V.z * vs;
        const float v2 = (vx * vx + vy * vy) + vz * vz;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int di = 0; di < 2; ++di) {
                    const float w = (wx[di] * wy[dy]) * wz[dz];
                    if (w == 0.f) continue;
                    const size_t nd = (size_t)((k + dz) * nxy + rr[dy] + ii[di]);
                    atomicAdd(m4 + nd, make_float4(w, w * vx, w * vy, w * vz));   // one vector reduction
                    atomicAdd(mk + nd, w * v2);
                }
    }
}

// add one sample's float sums to the FP64 window of its phase bin and clear them
__global__ void k_mom_fold(float4* __restrict__ m4, float* __restrict__ mk, double* __restrict__ mom,
                           double* __restrict__ mke, const int* bin, size_t nodes)
{
    const size_t b = (size_t)*bin;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nodes; q += (size_t)gridDim.x * blockDim.x) {
        const float4 m = m4[q];
        if (m.x == 0.f) continue;
        double* d = mom + 4 * (b * nodes + q);
        d[0] += (double)m.x;
        d[1] += (double)m.y;
        d[2] += (double)m.z;
        d[3] += (double)m.w;
        mke[b * nodes + q] += (double)mk[q];
        m4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        mk[q] = 0.f;
    }
}

__global__ void k_moments_phi(const double* phi, double* mphi, size_t n, const int* bin)
{
    mphi += (size_t)*bin * n;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        mphi[q] += phi[q];
}

P32 params(pic_ctx* c, int sp)
{
    P32 p;
    p.nx = c->nx; p.ny = c->ny; p.nz = c->nz; p.nxy = c->nx * c->ny;
    p.M = c->md_sub > 0 ? c->md_sub : 1;
    p.sp = sp;
    p.flags = c->flags;
    const double kq = c->qm[sp] * c->dt * c->dt / c->dx;
    p.kq = (float)kq;
    p.kqm = (float)(kq / (double)p.M);
    p.invM = (float)(1.0 / p.M);
    p.vs = (float)(c->dx / c->dt);
    p.inv_vs = (float)(c->dt / c->dx);
    p.hm = (float)c->hm[sp];
    p.pnull = (float)c->pnull[sp];
    p.nu_max = (float)c->nu_max[sp];
    p.de = (float)c->de[sp];
    p.n_gas = (float)c->n_gas;
    p.sig_n = (float)c->sig_n;
    p.eps_exc = (float)c->eps_exc;
    p.eps_ion = (float)c->eps_ion;
    p.mr2 = (float)((2.0 * kME) / kMAR);
    p.qk = (float)(1.0 / (4.0 * kPI * kEPS0) / (c->dx * c->dx));
    p.n_xs = c->n_xs;
    p.xs = c->xs32;
    p.key = c->key;
    p.step = c->d_step;
    p.gcell = c->gcell;
    p.goff = c->goff32;
    p.gr2 = c->gr2_32;
    p.gq = c->gq32;
    p.gtab = c->gtab32;
    p.gabs = c->gabs;
    p.cell_ng = c->cell_ng;
    p.cell_g = c->cell_g;
    p.E = c->e32;
    p.rq = c->rq;
    p.pos = (float4*)c->pos[sp];
    p.vel = (float4*)c->vel[sp];
    p.nslot = c->d_nslot;
    p.cnt = c->d_cnt;
    p.err = c->d_err;
    p.child = c->d_child;
    p.child_cap = (unsigned long long)c->child_cap;
    p.nch = c->d_nch;
    p.md_list = c->md_list[sp];
    p.md_n = c->d_lists + 2 * sp;
    p.md_next = c->md_next[sp];
    p.md_next_n = c->d_lists + 4 + sp;
    p.md_res = c->md_res[sp];
    p.md_rescap = (unsigned int)c->md_rescap;
    p.mcc_list = c->mcc_list[sp];
    p.mcc_n = c->d_lists + 2 * sp + 1;
    p.tstart = c->tstart[sp];
    p.tx = c->tile[0]; p.ty = c->tile[1]; p.tz = c->tile[2];
    p.ntx = c->ntile[0]; p.nty = c->ntile[1];
    p.ntiles = (long long)c->ntiles;
    p.halo = c->halo;
    p.wx = c->tile[0] + 1 + 2 * c->halo;
    p.wy = c->tile[1] + 1 + 2 * c->halo;
    p.wz = c->tile[2] + 1 + 2 * c->halo;
    return p;
}

}  // namespace

void launch_push32(pic_ctx* c)
{
    // this step's MD lists come from the last step; both species' MD particles
    // advance on a second branch while the bulk pushes run on the main stream
    k_md_rotate<<<64, 256, 0, c->stream>>>(c->md_list[0], c->md_next[0], c->md_list[1], c->md_next[1], c->d_lists);
    k_md_counts<<<1, 1, 0, c->stream>>>(c->d_lists);
    const P32 pe = params(c, 0), pi = params(c, 1);
    cudaEventRecord(c->ev_fork, c->stream);
    cudaStreamWaitEvent(c->aux, c->ev_fork, 0);
    k_md32<<<152 * 4, 64, 0, c->aux>>>(pe);
    k_md32<<<152 * 4, 64, 0, c->aux>>>(pi);
    cudaEventRecord(c->ev_join, c->aux);
    // both species of a tile in one block: one window, one flush
    const unsigned grid = (unsigned)(c->ntiles + kTailBlocks);
    const size_t win = sizeof(unsigned long long) * (size_t)pe.wx * pe.wy * pe.wz;
    k_push32<<<grid, kPushThreads, win, c->stream>>>(pe, pi);
    // the collision candidates of the two species, side by side
    cudaEventRecord(c->ev_fork, c->stream);
    cudaStreamWaitEvent(c->aux2, c->ev_fork, 0);
    k_mcc32<<<152 * 4, 256, 0, c->stream>>>(pe);
    k_mcc32<<<152 * 4, 256, 0, c->aux2>>>(pi);
    cudaEventRecord(c->ev_join2, c->aux2);
    cudaStreamWaitEvent(c->stream, c->ev_join2, 0);
    cudaStreamWaitEvent(c->stream, c->ev_join, 0);
    k_md_commit<<<64, 256, 0, c->stream>>>((float4*)c->pos[0], (float4*)c->vel[0], c->md_list[0], c->md_res[0],
                                           (float4*)c->pos[1], (float4*)c->vel[1], c->md_list[1], c->md_res[1],
                                           c->d_lists, (unsigned int)c->md_rescap,
                                           (c->flags & PIC_F_IONS_FROZEN) ? 1 : 0);
    c->launches += 8;
}

// The attribute belongs to the kernel, not to a run: it is raised to the
// largest window any tiling may ask for (an upper bound only; each launch's
// occupancy follows the window it actually takes), so that runs with
// different tilings in one process never lower it below each other's needs.
cudaError_t push32_set_window(pic_ctx*)
{
    return cudaFuncSetAttribute(k_push32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxWindowBytes);
}

void launch_deposit32(pic_ctx* c)
{
    for (int sp = 0; sp < 2; ++sp)
        k_deposit32<<<grid_for(c->cap[sp], 256, 152 * 8), 256, 0, c->stream>>>(c->nx, c->ny, (const float4*)c->pos[sp],
                                                                               c->d_nslot, sp, c->rq);
    c->launches += 2;
}

void launch_efield32(pic_ctx* c)
{
    const int bx = c->nx >= 32 ? 32 : c->nx, by = std::max(1, std::min(c->ny, 256 / bx));
    const dim3 grid((unsigned)((c->nx + bx - 1) / bx), (unsigned)((c->ny + by - 1) / by), (unsigned)(c->nz + 1));
    k_efield32<<<grid, dim3((unsigned)bx, (unsigned)by), 0, c->stream>>>(c->nx, c->ny, c->nz,
                                                                         (float)(1.0 / (2.0 * c->dx)), c->phi2, c->e32);
    c->launches += 1;
}

void launch_children32(pic_ctx* c)
{
    k_children32<<<64, 256, 0, c->stream>>>(c->nx, c->ny, c->d_child, c->d_nch, (unsigned long long)c->child_cap,
                                              c->d_nslot, c->d_next_id, (float4*)c->pos[0], (float4*)c->vel[0],
                                              (float4*)c->pos[1], (float4*)c->vel[1], c->cap[0], c->cap[1], c->rq,
                                              c->d_err, c->cell_ng, c->md_next[0], c->md_next[1], c->d_lists);
    k_children_finish32<<<1, 1, 0, c->stream>>>(c->d_nch, (unsigned long long)c->child_cap, c->d_nslot,
                                                c->d_next_id, c->cap[0], c->cap[1], c->d_step);
    c->launches += 2;
}

void launch_moments32(pic_ctx* c)
{
    for (int sp = 0; sp < 2; ++sp) {
        k_moments32<<<grid_for(c->cap[sp], 256, 152 * 8), 256, 0, c->stream>>>(
            c->nx, c->ny, (float)(c->dx / c->dt), (const float4*)c->pos[sp], (const float4*)c->vel[sp], c->d_nslot,
            sp, (float4*)c->mom32[sp], c->mom32[sp] + 4 * c->nodes);
        k_mom_fold<<<grid_for((int64_t)c->nodes, 256, 152 * 8), 256, 0, c->stream>>>(
            (float4*)c->mom32[sp], c->mom32[sp] + 4 * c->nodes, c->mom[sp], c->mke[sp], c->d_bin, c->nodes);
    }
    c->launches += 4;
}

void launch_moments_phi(pic_ctx* c)
{
    phi_sync_f64(c);
    k_moments_phi<<<grid_for((int64_t)c->nodes, 256, 152 * 4), 256, 0, c->stream>>>(c->phi, c->mphi, c->nodes,
                                                                                  c->d_bin);
    c->launches += 1;
}

}  // namespace pic

// Internal declarations of libpic: run context, device helpers and the kernel
// entry points shared between translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/pic.h"

namespace pic {

// physical constants (CODATA 2018)
constexpr double kQE = 1.602176634e-19;
constexpr double kEPS0 = 8.8541878128e-12;
constexpr double kME = 9.1093837015e-31;
constexpr double kAMU = 1.66053906660e-27;
constexpr double kKB = 1.380649e-23;
constexpr double kMAR = 39.948 * kAMU;
constexpr double kPI = 3.14159265358979323846;

constexpr int kWQ = 16384;      // fixed-point CIC weight units per axis
constexpr int kMaxG = 8;        // grains per MD cell
constexpr int kTab = 64 * 3;    // doubles per grain field table (4x4x4 nodes x 3)

// Philox counter third word: what the draws are for
enum Purpose : uint32_t {
    kPurMCC = 1, kPurDir = 2, kPurNeutral = 3, kPurChildDir = 4, kPurChildNeutral = 5,
    kPurInitPos = 10, kPurInitVel = 11   // the initial plasma (6-9: Coulomb pairing and scattering)
};

// error codes latched in ctx->d_err (first one wins)
enum DevErr : int { kErrNone = 0, kErrCapacity = PIC_ECAPACITY, kErrNonFinite = PIC_ENONFINITE };

// ionization product record: written by the push, numbered and appended later
struct ChildRec {
    uint32_t parent;
    int32_t cell;       // mixed: cell of the parent; fp64: unused
    double x[3];        // fp64: position (m); mixed: in-cell offsets
    double ve[3];       // new electron velocity (fp64: m/s; mixed: cells/step)
    double vi[3];       // new ion velocity
};

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: ten rounds of two 32x32->64 multiplies with a Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        // each 32 x 32 -> 64-bit product once, its low and high words
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        const uint32_t a0 = (uint32_t)p0, b0 = (uint32_t)(p0 >> 32);
        const uint32_t a1 = (uint32_t)p1, b1 = (uint32_t)(p1 >> 32);
        c = make_uint4(b1 ^ c.y ^ k.x, a1, b0 ^ c.w ^ k.y, a0);
    }
    return c;
}

// uniform on (0,1), exact in double
__device__ __forceinline__ double u01d(uint32_t u) { return ((double)u + 0.5) * 0x1p-32; }
__device__ __forceinline__ float u01f(uint32_t u) { return ((float)(u >> 8) + 0.5f) * 0x1p-24f; }

// ln x from +,-,*,/: x = m 2^e, m in [sqrt(1/2), sqrt(2)), ln m = 2 atanh((m-1)/(m+1))
// summed as an odd series to s^23 (Horner, no fused multiply-add in the fp64 unit)
__device__ __forceinline__ double ln_series(double x)
{
    int e;
    double m = frexp(x, &e);
    if (m < 0.70710678118654752440) { m = m * 2.0; e = e - 1; }
    const double s = (m - 1.0) / (m + 1.0);
    const double s2 = s * s;
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
    const double t1 = (double)e * 0.69314718055994530942;
    const double t2 = (2.0 * s) * p;
    return t1 + t2;
}

// Uniforms for one (particle id, step, purpose): successive Philox calls count
// in the fourth counter word; each call yields four 32-bit draws.
struct RStream {
    uint4 ctr;
    uint2 key;
    uint4 buf;
    int pos;
    __device__ RStream(uint32_t id, uint32_t step, uint32_t purpose, uint2 k)
        : ctr(make_uint4(id, step, purpose, 0u)), key(k), buf(make_uint4(0, 0, 0, 0)), pos(4) {}
    __device__ __forceinline__ uint32_t next()
    {
        if (pos == 4) { buf = philox4x32_10(ctr, key); ctr.w += 1u; pos = 0; }
        const uint32_t v = pos == 0 ? buf.x : pos == 1 ? buf.y : pos == 2 ? buf.z : buf.w;
        ++pos;
        return v;
    }
};

// ---------------------------------------------------------------- context
constexpr int kMaxDense = 1024;   // coarsest-level unknowns solved with a dense inverse
constexpr size_t kTailNodes = 2500;         // largest multigrid level held by one CTA

// constants of the graph solve's right-hand side and electrode values
struct SolveParams {
    double scale;       // rho_q units -> rho / eps0
    double inv_h2;
    double v_dc, v_rf, f_rf, phase, v_top, dt;
};

// device state of the mixed-precision (double-float) refinement
struct DfState {
    unsigned int cnt_head, cnt_res;   // block counters of the grid sums (wrap to 0)
    int sel;                          // buffer holding the current potential during a solve
    int more;                         // loop decision of the last residual
    int status;                       // PIC_OK, PIC_ENOTCONV or PIC_ENONFINITE after the last residual
    float b2;                         // ||h^2 b||^2 of the current solve
};

struct MGLevel {
    int nx, ny, nz;
    double h;
    size_t nodes;
    void* u = nullptr;   // T[nodes]
    void* f = nullptr;
    void* r = nullptr;
    int half = 0;        // > 0: u and f split by colour, node n of colour c at c * half + n / 2
};

}  // namespace pic

struct pic_ctx {
    // mesh and physics
    int nx, ny, nz;
    double dx, Lx, Ly, Lz;
    size_t nodes, cells;
    pic_electrodes el;
    double n_gas, t_gas, eps_exc, eps_ion, nu_max[2], de[2];
    int n_xs;
    int ng;
    int prec, flags, md_sub, sort_every, max_cycles;
    double W, dt, tol;
    uint64_t seed;
    uint32_t run_id;
    uint2 key;
    double qm[2], hm[2], pnull[2], sig_n;
    cudaStream_t stream;
    int64_t step;
    int64_t cap[2];
    int64_t child_cap;

    // particles: fp64 double4 {x,y,z,cell} / {vx,vy,vz,id}; mixed float4 {ox,oy,oz,cell bits} / {v (cells/step), id bits}
    void* pos[2] = {nullptr, nullptr};
    void* vel[2] = {nullptr, nullptr};
    void* pos_alt[2] = {nullptr, nullptr};
    void* vel_alt[2] = {nullptr, nullptr};
    unsigned long long* d_nslot = nullptr;   // [2] slots in use (live + holes since the last sort)
    unsigned long long* d_cnt = nullptr;     // [PIC_C_N]
    unsigned long long* d_live = nullptr;    // [2] live particles, counted on demand (pic_counts)
    int* d_err = nullptr;
    unsigned long long* d_nch = nullptr;     // children this step
    unsigned int* d_next_id = nullptr;
    pic::ChildRec* d_child = nullptr;
    unsigned int* md_list[2] = {nullptr, nullptr};   // mixed: slots of MD-region particles this step
    unsigned int* md_next[2] = {nullptr, nullptr};   // mixed: the same list being built for the next step
    float4* md_res[2] = {nullptr, nullptr};           // mixed: MD results (pos, vel pairs) until the join
    int64_t md_rescap = 0;
    unsigned int* mcc_list[2] = {nullptr, nullptr};  // mixed: slots of collision candidates this step
    unsigned int* d_lists = nullptr;                  // [md_n e, mcc_n e, md_n i, mcc_n i, next_n e, next_n i]

    // mesh arrays
    unsigned long long* rq = nullptr;        // int64 fixed-point charge per node
    double* phi = nullptr;                   // fp64 master potential
    double* phi_alt = nullptr;
    double* f64 = nullptr;                   // rho / eps0
    double* e64 = nullptr;                   // fp64: ex, ey, ez node arrays (3 * nodes)
    float4* e32 = nullptr;                   // mixed: {ex, ey, ez, 0} per node (V/m)
    double* d_norm = nullptr;                // [4] scratch norms

    // gas
    double* xs64 = nullptr;                  // 5 * n_xs
    float* xs32 = nullptr;

    // grains
    double* gpos = nullptr;                  // 3 ng (m)
    double* grad = nullptr;                  // ng
    int* gcell = nullptr;                    // 3 ng
    double* gq = nullptr;                    // ng (C)
    unsigned long long* gabs = nullptr;      // 2 ng
    double* gtab = nullptr;                  // ng * 192 (V/m per C)
    float* gtab32 = nullptr;
    float* gq32 = nullptr;                   // ng: Q (C)
    float* goff32 = nullptr;                 // 3 ng: centre offsets inside the grain's cell
    float* gr2_32 = nullptr;                 // ng: (radius / dx)^2
    int* cell_ng = nullptr;                  // cells
    int* cell_g = nullptr;                   // cells * 8

    // Coulomb collisions (PIC_F_COULOMB): per species, cell groups of slot indices
    double coul_log = 0.0;
    unsigned int* cs_end[2] = {nullptr, nullptr};        // cells: end of each cell's group
    unsigned int* cs_idx[2] = {nullptr, nullptr};        // capacity: slots grouped by cell
    unsigned long long* cs_key[2] = {nullptr, nullptr};  // capacity: pairing keys
    unsigned int* cs_cell[2] = {nullptr, nullptr};       // capacity: cell of each grouped slot
    unsigned int* cs_ord[2] = {nullptr, nullptr};        // capacity: slots grouped by cell, in key order

    // electron energy histogram (eepf_bins > 0): [k][bin], bins of eepf_de eV plus overflow
    unsigned long long* eepf = nullptr;
    int eepf_bins = 0;
    double eepf_de = 0.0;
    int64_t eepf_steps = 0;

    // sort scratch; the mixed path sorts by tile (tile[0] x tile[1] x tile[2]
    // cells, tile-major, cells row-major inside a tile), the FP64 path by cell
    unsigned int* hist = nullptr;            // nkeys + 1
    unsigned int* cursor = nullptr;          // nkeys + 1
    size_t nkeys = 0;                        // sort key range
    size_t nkeys_cap = 0;                    // keys the cursor buffer holds
    int64_t ntiles_cap = 0;                  // tiles the tstart buffers hold
    int tile[3] = {1, 1, 1};                 // mixed: tile edge in cells
    int ntile[3] = {1, 1, 1};                // mixed: tiles per axis
    int64_t ntiles = 0;
    int halo = 2;                            // mixed: deposit window margin around a tile, in cells
    int sort_order = 0;                      // mixed sort keys: 0 by cell inside the tile, 1 by tile only
    unsigned int* tstart[2] = {nullptr, nullptr};   // mixed: first slot of each tile after the last sort
                                                    // (ntiles + 1 entries; the last = particles sorted)
    std::vector<unsigned int*> scan_tmp;
    std::vector<size_t> scan_len;

    // multigrid
    std::vector<pic::MGLevel> mg;
    void* coarse_inv = nullptr;              // dense inverse of the coarsest level (T)
    int mg_tail = 0;                         // first level handled by the cluster kernel
    int cl_size = 1;                         // CTAs in that cluster
    int ex_level = -1;                       // level solved exactly by one cluster (-1: none)
    int ex_size = 1;                         // CTAs in that cluster
    void* ex_q = nullptr;                    // its x and y Fourier bases (T)
    void* ex_p = nullptr;                    // its Thomas pivots per mode (T)
    pic::SolveParams sp;
    unsigned int* d_iters = nullptr;         // graph solve: iterations of the last solve
    double* d_res = nullptr;                 // graph solve: relative residual of the last solve
    int* d_solve_flag = nullptr;             // graph solve: PIC_ENOTCONV / PIC_ENONFINITE latch
    uint32_t* d_step = nullptr;              // device copy of the step counter
    double* d_vb_last = nullptr;             // lower electrode value of the last solve
    float2* phi2 = nullptr;                  // mixed: potential as hi + lo floats, two buffers of nodes
    float2* f2 = nullptr;                    // mixed: h^2 rho / eps0 as hi + lo floats
    float* d_part = nullptr;                 // mixed: per-block partial sums
    pic::DfState* d_dfs = nullptr;
    unsigned long long* d_iter_total = nullptr;  // refinement iterations of all graph solves

    // CUDA graphs of one step, captured lazily on a private stream and
    // launched on the run's stream; variants by particle-buffer parity
    cudaStream_t cap_stream = nullptr;
    cudaStream_t aux = nullptr;              // second branch of the particle phase (MD, collisions)
    cudaStream_t aux2 = nullptr;             // third branch (the ion push beside the electron push)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
    int parity = 0;
    cudaGraphExec_t g_pre = nullptr, g_push[2] = {nullptr, nullptr}, g_solve = nullptr;
    cudaGraphExec_t g_post[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}}, g_mom[2] = {nullptr, nullptr};
    int n_pre = 0, n_push = 0, n_post[2] = {0, 0}, n_solve_head = 0, n_solve_body = 0, n_mom = 0;
    unsigned long long prof_iter0 = 0;

    // moments
    double* mom[2] = {nullptr, nullptr};     // nph * 4 * nodes each: [phase bin][node][n, n vx, n vy, n vz]
    double* mphi = nullptr;                  // nph * nodes
    double* mke[2] = {nullptr, nullptr};     // nph * nodes each: sum of n |v|^2
    float* mom32[2] = {nullptr, nullptr};    // mixed: one sample's float sums: float4 [node] {n, n v}, then float [node] n |v|^2
    double* d_oml = nullptr;                 // 6 per grain: hypothetical-charge estimate
    int64_t msteps = 0;
    int nph = 1;                             // rf phase bins of the moments
    double f_rf = 0.0, rf_phase = 0.0;
    int* d_bin = nullptr;                    // phase bin of the current sample
    unsigned long long* d_bsteps = nullptr;  // samples per phase bin
    int fine_n[3] = {0, 0, 0};
    size_t nfine = 0;
    double fine_h = 0.0, fine_o[3] = {0.0, 0.0, 0.0};
    double* fine[2] = {nullptr, nullptr};    // nfine * 4 each: [cube][count, sum vx, sum vy, sum vz]

    // measurement: events around push launches and solves while prof != 0
    int prof = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_push, ev_solve;
    int64_t prof_iters = 0;
    int64_t launches = 0;                    // kernels launched since pic_init

    // host-side status
    int64_t last_iters = 0;
    double last_res = 0.0;
    pic_status pending = PIC_OK;
    std::string err;
    std::vector<void*> allocs;
};

namespace pic {

// ---------------------------------------------------------------- kernel entry points
// particles_fp64.cu (built without fused multiply-add)
void launch_efield64(pic_ctx* c);
void launch_push64(pic_ctx* c);
void launch_children64(pic_ctx* c);
void launch_deposit64(pic_ctx* c);
void launch_moments64(pic_ctx* c);
void launch_grains(pic_ctx* c);                  // Q from counts, grain CIC into rq
void launch_grain_table(pic_ctx* c, int g);      // E of phi on grain g's 4x4x4 region nodes
// the initial plasma of species sp drawn from the seed (ids id0 ..), either layout
void launch_init_plasma(pic_ctx* c, int sp, int64_t n, uint32_t id0, double t_ev);
void launch_green_block(pic_ctx* c, int k, double* blk);   // phi near (0, 0, k) after a unit charge there
void launch_grain_tables_sup(pic_ctx* c, const double* blk, const int* plane);   // every grain's table from them
void launch_stage_particles(pic_ctx* c, int sp, const double* x, const double* v, const uint32_t* id, int64_t n,
                            int64_t q0, unsigned int* bad, unsigned int* max_id);   // caller particles into records

// particles_mixed.cu
void launch_efield32(pic_ctx* c);
void launch_push32(pic_ctx* c);
constexpr size_t kMaxWindowBytes = 96 * 1024;  // largest deposit window of the mixed push (shared memory)
cudaError_t push32_set_window(pic_ctx* c);     // lets the push take windows up to kMaxWindowBytes
void launch_children32(pic_ctx* c);
void launch_deposit32(pic_ctx* c);
void launch_moments32(pic_ctx* c);
void launch_moments_phi(pic_ctx* c);

// sort.cu
void sort_particles(pic_ctx* c, int sp);
void count_live(pic_ctx* c);                         // live records of both species into d_live
void scan_cells(pic_ctx* c, unsigned int* data);   // exclusive scan of one value per cell, in place

// diagnostics.cu (built without fused multiply-add)
void launch_eepf(pic_ctx* c);                       // add this step's electrons to the energy histogram
void launch_phase_bin(pic_ctx* c);                  // phase bin of this step's moment sample
void launch_fine(pic_ctx* c);                       // add this step's particles to the fine grid
void launch_oml(pic_ctx* c, int with_cx, double* out);   // 6 values per grain from the moment window

// coulomb.cu (built without fused multiply-add)
void launch_coulomb(pic_ctx* c);                    // binary Coulomb collisions of the step's particles
void launch_coulomb_fp64(pic_ctx* c);               // (its FP64 unit, built without fused multiply-add)
void launch_coulomb_mixed(pic_ctx* c);              // (its float unit)
size_t sort_scratch_setup(pic_ctx* c);

// poisson.cu
pic_status mg_setup(pic_ctx* c);
void launch_rhs(pic_ctx* c, double scale, double v_bot, double v_top, bool warm_shift);
void phi_sync_f64(pic_ctx* c);       // mixed: write the FP64 copy of the potential
void phi_from_f64(pic_ctx* c);       // mixed: potential from the FP64 copy
pic_status mg_solve(pic_ctx* c, double v_bot, double v_top, double tol, int max_iters, int* iters, double* res);
// graph solve pieces (enqueued on c->stream during capture)
void enqueue_solve_head(pic_ctx* c, double tol, int max_iters, cudaGraphConditionalHandle h);
void enqueue_solve_iteration(pic_ctx* c, double tol, int max_iters, cudaGraphConditionalHandle h);
void enqueue_solve_tail(pic_ctx* c);

// api.cu
void* dev_alloc(pic_ctx* c, size_t bytes);
int grid_for(int64_t n, int threads, int max_blocks);
// message returned by pic_last_error(NULL) for calls without a run context
void set_global_error(const char* msg);
// bracket one launch with events when measuring (begin returns the start event)
cudaEvent_t prof_begin(pic_ctx* c);
void prof_end(pic_ctx* c, cudaEvent_t start, bool push);

}  // namespace pic

#define PIC_CUDA_OK(expr) (cudaSuccess == (expr))

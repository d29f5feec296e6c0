/*
 * libpic — GB300 (sm_103a) PIC-MCC/PPPM particle cycle for electrons and Ar+
 * ions in an rf argon sheath around a fixed, self-consistently charging dust
 * cluster (Schleede et al., arXiv:1801.00972, Sec. III).
 *
 * The calls follow the paper's statement of the problem:
 *   - mesh, electrodes and rf drive (Sec. III, Fig. 2: cuboid of cubic cells,
 *     periodic laterally, metallic electrodes at both ends of the discharge
 *     axis, lower electrode driven sinusoidally, upper grounded).  Here the
 *     discharge axis is z: electrodes at z = 0 and z = nz*dx, periodic x, y.
 *   - gas (Sec. III: neutral argon reservoir of constant density at 300 K;
 *     Table I: e elastic, excitation, ionization; Ar+ elastic, charge
 *     exchange; cross sections supplied by the caller as tables);
 *   - grains (Sec. II-III: fixed positions and radii, perfect absorbers,
 *     charge zero at the start, changed by one super-particle charge per
 *     absorbed particle);
 *   - super-particles (Sec. III: weight W real particles each, leapfrog push
 *     of Eqs. 1-2 with time step dt, MD subcycling dt/40 near grains).
 *
 * Conventions for every call:
 *   - SI units (m, s, V, m^-3, K, eV where stated).
 *   - Pointers named *_host are host memory owned by the caller; the library
 *     copies inputs during the call and writes outputs of the stated length.
 *   - All device memory is allocated by pic_init and freed by pic_destroy.
 *   - Work is queued on the stream given to pic_init (NULL: the legacy default
 *     stream).  Calls that return data to the host synchronise that stream.
 *   - No call aborts or throws.  A failed call returns a non-zero pic_status
 *     and pic_last_error() describes it.  Errors that kernels detect
 *     (capacity overflow, non-finite values, particles faster than one box
 *     length per step) are latched on the device and returned by the next
 *     call that synchronises.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_ctx pic_ctx;

typedef enum {
    PIC_OK = 0,
    PIC_EINVAL = 1,      /* invalid argument or length mismatch             */
    PIC_ENOMEM = 2,      /* device or host allocation failed                */
    PIC_ECUDA = 3,       /* a CUDA runtime call failed                      */
    PIC_ECAPACITY = 4,   /* particle, child or fixed-point capacity exceeded */
    PIC_ENONFINITE = 5,  /* non-finite value or a particle moved > one box  */
    PIC_ENOTCONV = 6,    /* Poisson solve did not reach its tolerance       */
    PIC_ETIMEOUT = 7     /* a bounded device wait ran out                   */
} pic_status;

typedef enum { PIC_FP64 = 0, PIC_MIXED = 1 } pic_precision;

/* run flags (pic_run.flags) */
#define PIC_F_NO_MCC      1   /* no Monte Carlo collisions                       */
#define PIC_F_IONS_FROZEN 2   /* ions neither move nor collide (test use)        */
#define PIC_F_MOMENTS     8   /* accumulate node moments after every step        */
#define PIC_F_COULOMB    32   /* binary Coulomb collisions e-e, e-Ar+, Ar+-Ar+ (Table I)
                                 once per step, cell by cell, after the ionization
                                 products join: in-cell pairs in the order of a Philox
                                 key of (id, step), like pairs (0,1),(2,3),... with an odd
                                 count's first three as a triplet at half the time step,
                                 e-i pairs A[k] with B[k mod |B|] (A the larger group) at
                                 the smaller group's density; per pair tan(Theta/2) is
                                 normal with variance q^4 lnL n dt / (8 pi eps0^2 mu^2 u^3),
                                 the binary-collision model the paper cites (Sec. III) */
#define PIC_F_NO_GRAPH   16   /* pic_step launches kernels one by one and runs the
                                 Poisson loop from the host (for profilers that
                                 cannot see inside CUDA graphs); same results */
#define PIC_F_STAGE_COPY 128  /* pic_init copies the particle arrays to device
                                 scratch in chunks even where the device could read
                                 them in place (same records; for testing) */
#define PIC_F_F64_RESIDUAL 64 /* mixed precision only: the refinement residual of the
                                 Poisson solve in FP64 arithmetic instead of the
                                 double-float (two-float) arithmetic; the potential is
                                 still stored as two floats.  For measurement: same
                                 convergence, slower on this GPU's FP64 units */

/* Mesh: nx*ny*nz cubic cells of edge dx.  Phi and rho live on the cell corners
 * (Sec. III): nx*ny*(nz+1) nodes indexed (k*ny + j)*nx + i; x and y periodic,
 * node planes k = 0 and k = nz are the electrodes.  nx, ny >= 4, nz >= 2. */
typedef struct { int32_t nx, ny, nz; double dx; } pic_mesh;

/* phi(z=0, t) = v_dc + v_rf sin(2 pi f_rf t + phase); phi(z=nz*dx) = v_top
 * (Sec. II: 100 V amplitude at 13.56 MHz on the lower electrode, upper grounded). */
typedef struct { double v_dc, v_rf, f_rf, phase, v_top; } pic_electrodes;

/* Neutral argon (Sec. III, Table I).  xs_host holds 5 tables of n_xs values
 * (m^2) on uniform energy grids: electron elastic, excitation, ionization
 * (energy step de_e eV, energy = electron kinetic energy) and ion elastic,
 * charge exchange (step de_i eV, energy = ion energy relative to the neutral).
 * Linear interpolation between grid points; the last value beyond the grid.
 * nu_max_e / nu_max_i bound n_gas * sum(sigma) * v for the null-collision
 * method; a collision candidate occurs with probability 1 - exp(-nu_max dt). */
typedef struct {
    double n_gas, t_gas;          /* m^-3, K */
    double eps_exc, eps_ion;      /* eV */
    double nu_max_e, nu_max_i;    /* 1/s */
    double de_e, de_i;            /* eV */
    int32_t n_xs;
    const double* xs_host;        /* 5 * n_xs */
} pic_gas;

/* Grains (Sec. II-III): n fixed spheres, centres pos_host (3n, metres) and
 * radii radius_host (n, metres).  Each grain's cell must lie at least one cell
 * away from both electrodes; no cell may lie in more than 8 grains' MD regions. */
typedef struct { int32_t n; const double* pos_host; const double* radius_host; } pic_grains;

/* Super-particles and time stepping.  Initial particles are given per species
 * (0 = electrons, 1 = Ar+): positions x_host (3n, metres, inside the box),
 * velocities v_host (3n, m/s, taken as v at t = -dt/2) and unique ids (n).
 * capacity = particle slots per species (>= n; ionization adds particles). */
typedef struct {
    int64_t n[2];
    const double* x_host[2];
    const double* v_host[2];
    const uint32_t* id_host[2];
    int64_t capacity[2];
    double weight;                /* real particles per super-particle, W */
    double dt;                    /* s */
    int32_t md_sub;               /* MD substeps per step (Sec. III: 40) */
    int32_t sort_every;           /* counting-sort interval in steps (>= 1) */
    uint64_t seed;
    uint32_t run_id;
    int32_t prec;                 /* pic_precision */
    int32_t flags;                /* PIC_F_* */
    double tol;                   /* Poisson relative residual tolerance (e.g. 1e-10) */
    int32_t max_cycles;           /* Poisson refinement iterations per solve */
    double coulomb_log;           /* Coulomb logarithm lnL (> 0 with PIC_F_COULOMB) */
    int32_t eepf_bins;            /* > 0: accumulate the electron energy histogram of pic_eepf */
    double eepf_de_ev;            /* its bin width (eV) */
    int32_t mom_phases;           /* PIC_F_MOMENTS: > 1 also bins the moments by rf phase
                                     (pic_moments_phase); 0 or 1: rf averages only, in [0, 1024] */
    int32_t fine_n[3];            /* PIC_F_MOMENTS: fine diagnostic grid of fine_n[0] x fine_n[1] x
                                     fine_n[2] cubes of edge fine_h (Sec. IV.C: 200^3 cubes of
                                     0.08 dx over the MD region), lower corner fine_origin
                                     (metres), not periodic; all three 0 = off, else in [1, 1024] */
    double fine_h;
    double fine_origin[3];
} pic_run;

/* Create a run: copies every input to the device, deposits rho_0 (particles
 * plus grain charges, Sec. III), precomputes each grain's unit-charge mesh
 * field (Eq. 5) and solves phi_0 at t = 0.  On success *out owns the run.
 * The particle arrays are converted into the run's records on the device,
 * read in place where the device reads pageable host memory through the
 * host's page tables (a coherent CPU-GPU link), else copied in chunks of 2^24
 * particles; a particle outside the box or non-finite gives PIC_EINVAL after
 * the device has checked it (the other arguments are checked first, on the
 * host). */
pic_status pic_init(const pic_mesh* mesh, const pic_electrodes* el, const pic_gas* gas,
                    const pic_grains* grains, const pic_run* run, void* cuda_stream,
                    pic_ctx** out);

/* pic_init with the initial plasma drawn on the device from the run's seed
 * instead of host arrays (Sec. III starts from a plasma of given density and
 * electron and ion temperatures; the sampling rule is this library's):
 * run->n[0] electrons with ids 0 .. n[0]-1 and run->n[1] Ar+ ions with ids
 * n[0] .. n[0]+n[1]-1; run->x_host, v_host and id_host are ignored.  Particle
 * id p takes three uniforms at a time from its Philox stream (counter p,
 * step 0, purpose 10) for a point (u_x Lx, u_y Ly, u_z Lz), redrawn while it
 * lies within 1.5 radii of a grain (minimum image in x and y; at most 64
 * tries, then the last point is kept), and three standard normals (Marsaglia
 * polar method, purpose 11) times sqrt(t_ev[sp] e / m) for its velocity,
 * which is taken as v at t = -dt/2.  t_ev: 2 temperatures in eV (electrons,
 * ions), host memory.  Needs 1.5 * radius < dx for every grain and
 * n[0] + n[1] < 2^32; PIC_EINVAL otherwise.  Everything else as pic_init. */
pic_status pic_init_plasma(const pic_mesh* mesh, const pic_electrodes* el, const pic_gas* gas,
                           const pic_grains* grains, const pic_run* run, const double* t_ev, void* cuda_stream,
                           pic_ctx** out);

/* n_steps full time steps (Eqs. 1-6, MCC, absorption, deposit, Poisson), queued
 * on the run's stream.  Returns the status of the previous steps' solves. */
pic_status pic_step(pic_ctx* ctx, int32_t n_steps);

/* Autotune the counting-sort interval (the paper is silent on particle order;
 * it only affects speed: the deposit is an exact integer sum and the random
 * numbers are keyed on particle ids, so the physics does not depend on it).
 * Steps the run by at least steps_per_candidate steps (rounded up to whole
 * sort periods, at least two) for each interval in {2, 3, 4, 5, 6, 8, 10, 14,
 * 20}, timing each with CUDA events, and keeps the fastest.  The run advances
 * by all of these steps.  *chosen (may be NULL) receives the interval.
 * PIC_EINVAL for steps_per_candidate < 1; errors of the steps as pic_step. */
pic_status pic_tune_sort(pic_ctx* ctx, int32_t steps_per_candidate, int32_t* chosen);

/* Launch and layout choices of a run.  None of them changes a result: the
 * deposit is an exact integer sum and the random numbers are keyed on
 * particle ids, so any choice gives the same particles, charge and potential
 * bit for bit (the paper is silent on particle order and data layout).
 *   sort_every  counting-sort interval in steps (>= 1);
 *   tile        mixed precision: cells per tile along x, y, z; particles are
 *               sorted by tile and one thread block of the push takes a
 *               tile's particles (each edge in [1, min(mesh edge, 64)]);
 *   halo        mixed precision: margin in cells of the push's shared-memory
 *               deposit window around its tile, for the particles that drift
 *               out of the tile between sorts (in [0, 8]); the window of
 *               (tile + 1 + 2 halo) nodes per axis, 8 bytes each, must fit
 *               96 KB;
 *   order       mixed precision: 0 = particles sorted by cell inside each tile
 *               (the tile's cells row-major), 1 = by tile only (inside a tile
 *               they keep the order the sort meets them in: a cheaper sort,
 *               less locality in the push), 2 = by block of 2 x 2 x 2 cells
 *               inside the tile (in between).
 * The FP64 path uses sort_every only. */
typedef struct {
    int32_t sort_every;
    int32_t tile[3];
    int32_t halo;
    int32_t order;
} pic_tuning;

/* Current choices of a run (out: host). */
pic_status pic_get_tuning(const pic_ctx* ctx, pic_tuning* out);

/* Apply choices (in: host).  A new tile shape or margin synchronises the
 * run's stream, re-sorts both species at once and rebuilds the step graphs
 * at the next step.  PIC_EINVAL for values out of range. */
pic_status pic_set_tuning(pic_ctx* ctx, const pic_tuning* t);

/* Autotuner: times candidate choices on the run itself with CUDA events and
 * keeps the fastest, by coordinate search: tile shapes {8x8x8, 16x8x4, 8x8x4,
 * 16x8x8, 16x16x4, 32x8x4} (clipped to the mesh), then margins {1, 2, 3},
 * then the sort order {cell, tile, 2x2x2 blocks}, then sort intervals {2, 3, 4, 5, 6, 8, 10,
 * 14, 20}; each candidate runs at
 * least steps_per_candidate steps over whole sort periods after one warm-up
 * period, and the run advances by all of them.  With cache_path (may be NULL)
 * a cached entry for this (device name, mesh, particle count to two digits,
 * precision) is applied without timing; otherwise the result is added to the
 * cache file (see pic_tune_cache_store).  chosen (may be NULL, host) receives
 * the choices.  Errors of the steps as pic_step. */
pic_status pic_tune(pic_ctx* ctx, int32_t steps_per_candidate, const char* cache_path, pic_tuning* chosen);

/* The autotuner's cache file, host only (no GPU): a JSON object with one
 * member per line, "key": {"sort_every": S, "tile": [X, Y, Z], "halo": H,
 * "order": O} (an entry without "order" reads as order 0).
 * load: PIC_OK and *out when the file holds `key`, else PIC_EINVAL.  store:
 * adds or replaces `key` (no '"' or newline in it) and rewrites the file
 * through a temporary file in the same directory; PIC_EINVAL when it cannot
 * be written. */
pic_status pic_tune_cache_load(const char* path, const char* key, pic_tuning* out);
pic_status pic_tune_cache_store(const char* path, const char* key, const pic_tuning* t);

/* The particle half of one step: CIC gather of -grad phi (Eq. 4), leapfrog push
 * (Eqs. 1-2) with MD subcycling and the PPPM correction (Eqs. 5-6) near grains,
 * electrode and grain absorption, null-collision MCC with ionization products,
 * grain charge update and the fixed-point CIC deposit of rho_{k+1}; then
 * step += 1.  Does not solve for phi. */
pic_status pic_advance(pic_ctx* ctx);

/* Solve Eq. 3 for the current rho with the electrode values at t = step*dt,
 * warm-started from the current phi.  Optional outputs: refinement iterations
 * used and final relative residual ||b - A phi|| / ||b|| (host pointers). */
pic_status pic_solve(pic_ctx* ctx, int32_t* iterations, double* rel_residual);

/* Grain state: n_abs_host (2*n: electrons, ions absorbed, cumulative, exact)
 * and q_host (n: Q = e W (N_ion - N_e), coulomb). Either may be NULL. */
pic_status pic_grain_charges(pic_ctx* ctx, int64_t* n_abs_host, double* q_host);

/* Live particle counts (2) and event counters (PIC_C_N, cumulative). */
#define PIC_C_LOST_BOT_E 0
#define PIC_C_LOST_BOT_I 1
#define PIC_C_LOST_TOP_E 2
#define PIC_C_LOST_TOP_I 3
#define PIC_C_ABS_E      4
#define PIC_C_ABS_I      5
#define PIC_C_E_EL       6
#define PIC_C_E_EXC      7
#define PIC_C_E_ION      8
#define PIC_C_I_EL       9
#define PIC_C_I_CX      10
#define PIC_C_ERR       11
#define PIC_C_PUSHED    12   /* live particles processed by the push kernels */
#define PIC_C_N         13
pic_status pic_counts(pic_ctx* ctx, int64_t* n_live_host /* 2 */, int64_t* counters_host /* PIC_C_N */);

/* Electron energy histogram for the EEPF (Sec. IV.A, Fig. 3), accumulated
 * every step after the collisions when run->eepf_bins > 0: counts[k][b] is the
 * number of electron super-particles in cell plane k (z from k dx to (k+1) dx)
 * with energy eps = (m_e/2)|v|^2/e in [b de, (b+1) de) eV, b < eepf_bins, and
 * column eepf_bins counts the energies beyond, summed over the steps since
 * pic_init or the last reset.  len = nz * (eepf_bins + 1); *steps (may be NULL)
 * receives the number of steps summed.  reset != 0 clears after reading.
 * The EEPF of a slab is g(eps) = sum_k counts[k][b] W / (V de sqrt(eps)) at
 * the bin centres (V the slab volume, W the weight).
 * PIC_EINVAL for a wrong len or when the histogram is off. */
pic_status pic_eepf(pic_ctx* ctx, int64_t* counts, size_t len, int64_t* steps, int32_t reset);

/* Two-Maxwellian fit of an EEPF histogram (one slab, nbins counts without the
 * overflow column): g(eps) = A_l exp(-eps/T_l) + A_h exp(-eps/T_h) over the bin
 * centres in [e_lo_ev, e_hi_ev], g_b = counts_b / (de sqrt(eps_b)), as the
 * paper fits its bulk EEPF (Sec. IV.A: T_l = 0.31 eV, T_h = 2.32 eV there).
 * fit[4] receives T_l, T_h (eV), A_l, A_h; a single temperature gives T_l =
 * T_h and A_l = 0.  Host only, touches no GPU.  PIC_EINVAL for bad arguments
 * or fewer than 4 non-empty bins in range. */
pic_status pic_eepf_fit(const int64_t* counts, int32_t nbins, double de_ev, double e_lo_ev, double e_hi_ev,
                        double* fit);

/* Window averages since the last reset (needs PIC_F_MOMENTS), sampled after
 * every step (positions at t = step dt, the velocities of the step, phi of the
 * step's solve): what 0 phi (V, nodes), 1 n_e, 2 n_i (m^-3, nodes, CIC
 * weights), 3 flux_e, 4 flux_i (m^-2 s^-1, 3 per node, node-major), 5 T_e,
 * 6 T_i (eV per node: (m/3e)(<v^2> - |<v>|^2) of the window's CIC-weighted
 * velocities, 0 where no particle reached the node).  len = number of doubles
 * in out_host.  reset != 0 then clears every moment window
 * (rf average, phase bins and the fine grid). */
pic_status pic_moments(pic_ctx* ctx, int32_t what, double* out_host, size_t len, int32_t reset);

/* The same averages over the samples of one rf phase bin (Sec. IV.C: electron
 * fluxes resolved in rf phase).  The sample after step s falls in bin
 * floor(frac(f_rf s dt + phase / 2 pi) * mom_phases), i.e. the electrode phase
 * modulo 2 pi cut into mom_phases equal bins from 0.  *steps_out (optional) =
 * samples in that bin.  PIC_EINVAL for a bin out of range or an empty bin. */
pic_status pic_moments_phase(pic_ctx* ctx, int32_t what, int32_t bin, double* out_host, size_t len,
                             int64_t* steps_out);

/* Hypothetical charge of every grain with no other grains around (Sec. IV.B,
 * Fig. 7): the orbital-motion-limited balance of electron and ion currents,
 * with (with_cx != 0) the charge-exchange ion current 0.1 (e phi/T_i)^2
 * lambda_D/l_i of the weakly collisional model of Khrapak et al. (2005), from
 * the window's n, <v>, <v^2> CIC-interpolated to the grain centre; l_i from
 * n_gas and the charge-exchange table at 3/2 T_i.  out_host: 6 doubles per
 * grain, Q = 4 pi eps0 a phi (C), phi (V), n_e, n_i (m^-3), T_e, T_i (eV); Q
 * and phi are NaN where a local density or temperature is not positive.
 * Needs PIC_F_MOMENTS and a non-empty window; len = 6 * grains. */
pic_status pic_oml_charges(pic_ctx* ctx, int32_t with_cx, double* out_host, size_t len);

/* Window averages on the fine grid (needs fine_n): what 1 n_e, 2 n_i (m^-3 per
 * fine cube), 3 flux_e, 4 flux_i (m^-2 s^-1, 3 per cube); cube (i, j, k) at
 * index (k * fine_n[1] + j) * fine_n[0] + i holds the particles with
 * fine_origin + (i, j, k) fine_h <= x < fine_origin + (i+1, j+1, k+1) fine_h. */
pic_status pic_fine_moments(pic_ctx* ctx, int32_t what, double* out_host, size_t len);

/* Parity and inspection hooks (same conventions; lengths are checked). */
pic_status pic_get_particles(pic_ctx* ctx, int32_t species, double* x_host, double* v_host,
                             uint32_t* id_host, int64_t cap, int64_t* n_out);
pic_status pic_get_rho(pic_ctx* ctx, int64_t* rho_q_host, size_t len); /* units e W 2^-42 per node */
pic_status pic_get_phi(pic_ctx* ctx, double* phi_host, size_t len);
pic_status pic_set_phi(pic_ctx* ctx, const double* phi_host, size_t len);
pic_status pic_get_grain_table(pic_ctx* ctx, double* tab_host, size_t len); /* n*64*3 */
pic_status pic_set_grain_table(pic_ctx* ctx, const double* tab_host, size_t len);
pic_status pic_set_grain_counts(pic_ctx* ctx, const int64_t* n_abs_host, size_t len);
int64_t    pic_step_index(const pic_ctx* ctx);

/* Measurement: from pic_profile(ctx, 1) on, CUDA events recorded on the run's
 * stream bracket every push-kernel launch and every Poisson solve; pic_profile(ctx, 0)
 * stops recording.  pic_profile_read returns the summed device time (ms) and
 * counts since recording started, and the number of kernels the library has
 * launched since pic_init (all kinds).  Any pointer may be NULL. */
pic_status pic_profile(pic_ctx* ctx, int32_t enable);
pic_status pic_profile_read(pic_ctx* ctx, double* push_ms, int64_t* push_launches, double* solve_ms,
                            int64_t* solves, int64_t* solve_iterations, int64_t* kernels_launched);

/* Batched ensemble: n independent runs (seeds, rf phases, pressures, grain
 * clusters, meshes of different sizes), each described by element r of the
 * argument arrays exactly as for pic_init.  The batch gives every run its own
 * CUDA stream; pic_batch_step queues each run's step graphs on its stream, so
 * the runs execute concurrently on the GPU, and returns after all of them
 * (the first failing run's status).  Results of a run are identical to the
 * same run made alone with pic_init/pic_step.  pic_batch_run lends run r's
 * context to the query calls (do not pass it to pic_destroy). */
typedef struct pic_batch pic_batch;
pic_status pic_batch_init(int32_t n, const pic_mesh* meshes, const pic_electrodes* els, const pic_gas* gases,
                          const pic_grains* grains, const pic_run* runs, pic_batch** out);
pic_status pic_batch_step(pic_batch* b, int32_t n_steps);
pic_ctx*   pic_batch_run(pic_batch* b, int32_t r);
void       pic_batch_destroy(pic_batch* b);

/* Poisson solve that allocates nothing.  The paper has no counterpart: this is
 * a service for callers that cannot call cudaMalloc, such as a host application
 * whose own memory manager has already reserved the device memory (an extra
 * cudaMalloc fails or escapes its accounting), or a time-critical loop that must
 * avoid cudaMalloc/cudaFree because they synchronise the whole device.
 *
 * It solves the discrete Poisson equation of pic_solve, -lap(phi) = rho/eps0
 * with the 7-point stencil, periodic in x and y, Dirichlet node planes k = 0
 * (v_bot) and k = nz (v_top), by multigrid V(2,2) cycles inside FP64 residual
 * refinement (mixed: FP32 cycles; FP64: FP64 cycles), for a mesh of at most
 * 131072 nodes (nx*ny*(nz+1)).  Its coarse levels differ from pic_solve's:
 * the mesh is halved while nx and ny are divisible by 4 and nz is even and
 * at least 4, and the coarsest level is smoothed by up to 2000 red-black
 * Gauss-Seidel sweeps in one thread block (pic_solve solves its coarse level
 * exactly).  Meshes larger than 131072 nodes, or whose coarsest level has
 * more than 4096 nodes, return PIC_EINVAL.  The caller passes device
 * pointers:
 *   rho_q_dev  int64 fixed-point charge per node, as pic_get_rho returns it;
 *   scale      factor turning rho_q into rho/eps0 (for a run of weight W:
 *              e W / dx^3 * 2^-42 / eps0);
 *   phi_dev    FP64 potential per node: the start value on entry (e.g. zeros or
 *              the previous solution, even one with other electrode values),
 *              the solution on return; the electrode planes are set to v_bot
 *              and v_top.
 * prec is PIC_FP64 or PIC_MIXED; tol, max_iters, iterations and rel_residual
 * mean what they mean for pic_solve.  Work runs on cuda_stream (NULL: default).
 * Every call reads norms back to the host and synchronises cuda_stream, so it
 * must not be made while that stream is being captured into a CUDA graph.
 *
 * The working set lives in one fixed device array of about 6.3 MB inside the
 * library, which every GPU that loads the library holds until the process
 * exits.  The first call on a device looks up that array's device address
 * (once per device, for the current device).  Every call reuses the same
 * array and overwrites what the previous call left there, so calls that
 * overlap on the GPU (from several host threads or streams at once) race and
 * must be serialised by the caller. */
pic_status pic_solve_noalloc(int32_t nx, int32_t ny, int32_t nz, double dx, const int64_t* rho_q_dev, double scale,
                             double v_bot, double v_top, double* phi_dev, int32_t prec, double tol,
                             int32_t max_iters, int32_t* iterations, double* rel_residual, void* cuda_stream);

const char* pic_last_error(const pic_ctx* ctx);   /* NULL ctx: last pic_init failure */
void pic_destroy(pic_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif

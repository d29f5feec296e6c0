/*
 * Oracle for the PIC-MCC/PPPM particle cycle of "Plasma flow around and
 * charge distribution of a dust cluster in a rf discharge" (Schleede et al.,
 * arXiv:1801.00972), Sec. III.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, FP64 CPU restatement of
 * the method, used to check the CUDA library.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header or constant table with the CUDA library.
 *
 * Units are SI throughout: positions in metres, velocities in m/s, charges in
 * coulomb, potentials in volt.  Species 0 = electrons, 1 = Ar+ ions.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* flags */
#define ORC_NO_MCC      1   /* skip Monte Carlo collisions                     */
#define ORC_IONS_FROZEN 2   /* ions neither move nor collide (test-only)       */
#define ORC_MOMENTS     8   /* accumulate node moments every step              */
#define ORC_COULOMB    32   /* binary Coulomb collisions e-e, i-i, e-i (Table I) */
#define ORC_EEPF       64   /* electron energy histogram per cell plane, every step */

typedef struct {
    int32_t nx, ny, nz, md_sub;      /* cells; MD subcycles per step (Sec. III: 40) */
    double  dx, dt, weight;          /* cell edge, time step, real particles per super-particle */
    double  v_dc, v_rf, f_rf, phase, v_top;   /* phi(z=0,t) = v_dc + v_rf sin(2 pi f t + phase) */
    double  n_gas, t_gas;            /* neutral density (m^-3) and temperature (K) */
    double  eps_exc, eps_ion;        /* excitation / ionization thresholds (eV) */
    double  nu_max_e, nu_max_i;      /* null-collision frequency bounds (1/s) */
    double  de_e, de_i;              /* energy step of the cross-section tables (eV) */
    int32_t n_xs, n_grains;
    const double* xs;                /* 5*n_xs: e_el, e_exc, e_ion, i_el, i_cx (m^2) */
    const double* gpos;              /* 3*n_grains, metres */
    const double* grad;              /* n_grains, metres */
    uint64_t seed;
    uint32_t run_id;
    int32_t  flags;
    int64_t  n_init[2];
    const double*   x_init[2];       /* 3*n per species */
    const double*   v_init[2];       /* 3*n per species */
    const uint32_t* id_init[2];      /* n per species */
    double   coulomb_log;            /* Coulomb logarithm of the binary collisions (ORC_COULOMB) */
    int32_t  eepf_bins;              /* ORC_EEPF: energy bins of width eepf_de_ev, plus one overflow bin */
    double   eepf_de_ev;
    int32_t  mom_phases;             /* ORC_MOMENTS: > 1 also bins the node moments by rf phase */
    int32_t  fine_n[3];              /* ORC_MOMENTS: fine diagnostic grid of fine_n[0..2] cells of */
    double   fine_h;                 /*   edge fine_h (all three > 0 switch it on), lower corner  */
    double   fine_origin[3];         /*   fine_origin (metres); not periodic                       */
    double   t_init_ev[2];           /* species with n_init > 0 and x_init NULL: sampled here from the
                                        seed (uniform in the box outside 1.5 grain radii, Maxwellian at
                                        t_init_ev), ids 0..n_e-1 for electrons, n_e.. for ions */
} orc_cfg;

typedef struct orc_sim orc_sim;

/* counters returned by orc_get_counters (cumulative since creation) */
enum { ORC_C_LOST_BOT_E, ORC_C_LOST_BOT_I, ORC_C_LOST_TOP_E, ORC_C_LOST_TOP_I,
       ORC_C_ABS_E, ORC_C_ABS_I, ORC_C_E_EL, ORC_C_E_EXC, ORC_C_E_ION,
       ORC_C_I_EL, ORC_C_I_CX, ORC_C_ERR, ORC_C_N };

orc_sim* orc_create(const orc_cfg* cfg);           /* deposits rho_0 and solves phi_0 */
void     orc_destroy(orc_sim* s);
int      orc_advance(orc_sim* s);                   /* particles, grains, children, deposit; step += 1 */
int      orc_solve(orc_sim* s);                     /* phi from rho at t = step*dt */
int      orc_step(orc_sim* s);                      /* advance + solve */
void     orc_coulomb(orc_sim* s);                   /* one Coulomb collision pass at the current step */
/* electron counts per (cell plane k, energy bin), nz * (eepf_bins + 1), summed over the steps since
 * creation; returns the number of steps summed */
int64_t  orc_get_eepf(const orc_sim* s, int64_t* counts);

int64_t  orc_count(const orc_sim* s, int sp);
void     orc_get_particles(const orc_sim* s, int sp, double* x, double* v, uint32_t* id);
void     orc_get_rho(const orc_sim* s, int64_t* rq);
void     orc_get_phi(const orc_sim* s, double* phi);
void     orc_set_phi(orc_sim* s, const double* phi);
void     orc_get_grains(const orc_sim* s, int64_t* n_abs /* 2*ng: e,i */, double* q);
void     orc_get_gtab(const orc_sim* s, double* tab /* ng*64*3 */);
void     orc_set_gtab(orc_sim* s, const double* tab);
void     orc_get_counters(const orc_sim* s, int64_t* c /* ORC_C_N */);
int64_t  orc_step_index(const orc_sim* s);
uint32_t orc_next_id(const orc_sim* s);
/* what: 0 phi, 1 n_e, 2 n_i, 3 flux_e (3 per node), 4 flux_i, 5 T_e, 6 T_i (eV, the
 * temperature of the window's node-weighted velocity distribution); window averages */
int      orc_moments(const orc_sim* s, int what, double* out);
/* the same for the samples of rf phase bin `bin` only; *steps = samples in that bin */
int      orc_moments_phase(const orc_sim* s, int what, int bin, double* out, int64_t* steps);
/* fine grid, what: 1 n_e, 2 n_i (per fine cell), 3 flux_e, 4 flux_i (3 per fine cell) */
int      orc_fine_moments(const orc_sim* s, int what, double* out);
void     orc_reset_moments(orc_sim* s);
/* OML surface potential (V) of an isolated sphere in a plasma of densities ne,
 * ni (m^-3) and temperatures te, ti (eV) of electrons and Ar+, with the
 * charge-exchange ion flux term 0.1 (e phi / T_i)^2 lambda_D / l_i given by
 * lam_over_l = lambda_D / l_i (0: collisionless OML); NaN if a density or a
 * temperature is not positive.  Parity partially pinned: the collisionless
 * balance against its closed forms, and the charge-exchange term through the
 * potential a chosen lam_over_l balances and its sign.  Its 0.1 coefficient
 * is the cited model's, with no independent check here (parity unpinned for
 * that coefficient).  orc_oml_charges' lambda_D / l_i is pinned against the
 * textbook Debye length and sigma_cx at 3/2 T_i. */
double   orc_oml_potential(double ne, double ni, double te, double ti, double lam_over_l);
/* per grain 6 values from the moment window: Q = 4 pi eps0 a phi (C), phi (V),
 * and the local n_e, n_i (m^-3), T_e, T_i (eV) at the grain centre; with_cx
 * adds the charge-exchange ion flux.  Returns -1 without ORC_MOMENTS samples. */
int      orc_oml_charges(const orc_sim* s, int with_cx, double* out);
/* test helpers: field acting on a particle at p (Eqs. 4-6, with the MD
 * correction when p's cell is in an MD region); set the grains' absorbed
 * counts, which redeposits rho and re-solves phi at the current time */
int      orc_field_at(orc_sim* s, const double p[3], double E[3]);
void     orc_set_grain_counts(orc_sim* s, const int64_t* n_abs /* 2*ng */);

/* host threads of the parallel loops (1 without OpenMP); set n (0: all cores) */
int      orc_threads(void);
void     orc_set_threads(int n);

/* stand-alone pieces, used by the tests that pin the oracle */
void     orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double   orc_ln(double x);
int      orc_poisson(int nx, int ny, int nz, double dx, const double* f, double v_bot,
                     double v_top, double* phi);
void     orc_efield(int nx, int ny, int nz, double dx, const double* phi,
                    double* ex, double* ey, double* ez);
void     orc_iso_dir(uint32_t id, uint32_t step, uint32_t purpose, const uint32_t key[2], double out[3]);
void     orc_gauss3(uint32_t id, uint32_t step, uint32_t purpose, const uint32_t key[2], double out[3]);

#ifdef __cplusplus
}
#endif
#endif

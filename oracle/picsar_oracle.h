/*
 * picsar_oracle.h -- FP64 CPU oracle for the PICsar time step (arXiv 1407.1810).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and oracle/picsar_oracle.c are a plain,
 * slow, single-threaded restatement of the method, written from the paper, used
 * to check the GPU library.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code with the GPU library.
 *
 * Conventions (the paper's Lorentz-Heaviside units, Sec. 2, with c = 1):
 *   grid: nr x nth cells; nodes i = 0..nr (radial), j = 0..nth (meridional);
 *   grid coordinate x = (x1, x2), node (i, j) sits at r = f_r(i), theta = f_th(j)
 *   (Sec. 3.2).  Field components live at the staggered points of Eq. (offseteq).
 *   Particles carry x1, x2, momentum u = gamma v in the local spherical basis
 *   (u_r, u_th, u_ph), and a signed macro-charge qw; mass = |qw| / q_over_m.
 */
#ifndef PICSAR_ORACLE_H
#define PICSAR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_R_LINEAR = 0, ORC_R_LOG = 1 };
enum { ORC_TH_LINEAR = 0, ORC_TH_EQUAL_AREA = 1 };
enum { ORC_ABSORB_NONE = 0, ORC_ABSORB_LINEAR = 1, ORC_ABSORB_QUADRATIC = 2 };
enum { ORC_VAC_NONE = 0, ORC_VAC_MONOPOLE = 1, ORC_VAC_MONOPOLE_ROTATOR = 2,
       ORC_VAC_UNIFORM_BZ = 3, ORC_VAC_DIPOLE_COROT = 4, ORC_VAC_DIPOLE_ROTATOR = 5 };
enum { ORC_INJECT_OFF = 0, ORC_INJECT_FIXED = 1, ORC_INJECT_VARIABLE = 2 };
enum { ORC_VAY = 0, ORC_BORIS = 1 };

typedef struct orc_params {
  int32_t nr, nth;          /* cells */
  double r_min, r_max;      /* inner / outer conductor radius; r_min is r0 */
  int32_t r_map, th_map;    /* stretching functions, Sec. 3.2 */
  double dt;                /* time step (c = 1) */
  int32_t n_filt;           /* 1-2-1 passes, App. B */
  int32_t absorb_cells;     /* lossy layer width Delta L in cells, Sec. 3.4.1 */
  int32_t absorb_profile;   /* ORC_ABSORB_* */
  double absorb_sigma_max;  /* sigma* at the outer edge; <= 0: 2/dL (linear), 3/dL (quadratic) */
  int32_t vacuum;           /* ORC_VAC_* analytic "initial" field, Sec. 5.2 / 4.3 */
  double b0;                /* field at r0 */
  double omega;             /* final angular velocity; light cylinder R_l = 1/omega */
  double t_spin;            /* linear spin-up time, Sec. 5.2 */
  int32_t inject;           /* ORC_INJECT_*: surface injection, Sec. 5.3 */
  int32_t pairs_per_cell;   /* FIXED: pairs per surface cell per step; VARIABLE: the cap */
  double f_inj;             /* injection multiplier, Eq. (volinjeq) */
  int32_t pusher;           /* ORC_VAY | ORC_BORIS, Sec. 2 */
  double q_over_m;          /* |q|/m of every species (pair plasma) */
  int32_t inject_smooth;    /* 1-2-1 passes over sigma_j along theta before injecting */
  double inject_q;          /* VARIABLE: |charge| of each injected particle */
  uint64_t inject_seed;     /* VARIABLE: seed of the stochastic rounding (SplitMix64) */
} orc_params;

typedef struct orc_sim orc_sim;

/* lifetime */
orc_sim *orc_create(const orc_params *p);
void orc_destroy(orc_sim *s);
int orc_last_error(const orc_sim *s);      /* 0 or a negative code (see .c) */

/* grid maps and metric (Sec. 3.2, Eq. linearea) */
double orc_f_r(const orc_sim *s, double x1);
double orc_f_r_inv(const orc_sim *s, double r);
double orc_f_th(const orc_sim *s, double x2);
double orc_f_th_inv(const orc_sim *s, double th);
double orc_courant_dt(const orc_params *p, double courant);

/* particles (appended; ids given explicitly, or -1 for 0..n-1 continuing next_id) */
void orc_load_particles(orc_sim *s, int64_t n, const double *x1, const double *x2,
                        const double *ur, const double *uth, const double *uph,
                        const double *qw, const int64_t *id);
int64_t orc_num_particles(const orc_sim *s);
void orc_get_particles(const orc_sim *s, double *x1, double *x2, double *ur,
                       double *uth, double *uph, double *qw, int64_t *id);
void orc_set_clock(orc_sim *s, int64_t step, int64_t next_id);
int64_t orc_get_step(const orc_sim *s);

/* fields: out/in = 6 planes [E_r, E_th, E_ph, B_r, B_th, B_ph] of (nr+1) x (nth+1),
 * row-major [i][j]; entries outside a component's staggered range are 0. */
void orc_get_fields(const orc_sim *s, double *out6);
void orc_set_fields(orc_sim *s, const double *in6);
/* the same layout, plasma plus analytic field at time step * dt (Sec. 5.2) */
void orc_get_fields_total(const orc_sim *s, double *out6);
/* fluxes F_r, F_th, F_ph of the last step (after filtering): 3 planes of
 * (nr+2g+1) x (nth+1), row index i+g, g = n_filt+2. */
int32_t orc_ghost(const orc_sim *s);
void orc_get_flux(const orc_sim *s, double *out3);

/* one or more full time steps */
void orc_step(orc_sim *s, int32_t nsteps);
/* the particle part of one step (no field update, clock unchanged) */
void orc_particles_only(orc_sim *s);
/* field-only leapfrog with zero current (Appendix A), used by the field tests */
void orc_field_step(orc_sim *s, int32_t nsteps);

/* single-particle building blocks, exposed for the tests */
void orc_vacuum_fields(const orc_sim *s, double x1, double x2, double t, double E[3], double B[3]);
void orc_gather(const orc_sim *s, double x1, double x2, double t, double E[3], double B[3]);
void orc_push(int32_t pusher, double qmdt, const double E[3], const double B[3], double u[3]);
/* deposit one straight grid-coordinate path a->b of charge qw into caller arrays
 * laid out like orc_get_flux (F_r, F_th planes only); returns 0 or -1 (> 1 cell). */
int orc_deposit_path(const orc_sim *s, double qw, double a1, double a2, double b1, double b2,
                     double *fr, double *fth);
void orc_filter_pass(const orc_sim *s, double *f, int32_t half_j, int32_t sign);

/* diagnostics */
void orc_node_charge(const orc_sim *s, int32_t absolute, double *q);  /* (nr+2g+1) x (nth+1) */
void orc_gauss_snapshot(orc_sim *s);
double orc_gauss_residual(const orc_sim *s);
double orc_field_energy(const orc_sim *s);
double orc_kinetic_energy(const orc_sim *s);
void orc_divb(const orc_sim *s, double *out); /* nr x nth cells: flux of B out of each cell */
/* radial Poynting flux through the sphere of each node radius (total field at
 * time t); out: nr + 1 values, 0 at i = 0 and nr */
void orc_luminosity(const orc_sim *s, double t, double *out);
/* live, deleted, injected, next_id, capped (VARIABLE injection: cells whose
 * pair count was cut to pairs_per_cell) */
void orc_counters(const orc_sim *s, int64_t *out5);
/* R15: ties of the azimuth branch at the polar axis met so far, and hints
 * (step, id -> sign) that fix the branch of the ties they list */
int64_t orc_axis_ties(const orc_sim *s);
void orc_set_axis_hints(orc_sim *s, int64_t n, const int64_t *steps, const int64_t *ids, const int32_t *signs);
/* R13: stochastic-rounding draws within 1e-4 n_j of the threshold so far */
int64_t orc_inject_ties(const orc_sim *s);
/* output number n + 1 of the SplitMix64 stream seeded with `seed` */
uint64_t orc_splitmix64(uint64_t seed, uint64_t n);

#ifdef __cplusplus
}
#endif
#endif

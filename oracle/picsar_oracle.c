/*
 * picsar_oracle.c -- FP64 CPU oracle for the PICsar time step (arXiv 1407.1810).
 *
 * TEST INFRASTRUCTURE ONLY.  A plain, slow, single-threaded restatement of the
 * method, written from the paper so that a reader can check each function
 * against the section or equation it cites.  The GPU library is checked against
 * it; the two share no code.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file.
 *
 * Readings of the paper where it is silent (each also listed in the project's
 * design notes):
 *   R1 Gauss law in Lorentz-Heaviside units, integral form: G - Q per dual cell.
 *   R2 Field gather: bilinear in grid coordinates from each staggered component;
 *      below/above the polar axis, half-integer-j values continue axisymmetrically
 *      (B_r even; E_th, B_ph odd); radial values outside the conductors are 0.
 *      Inside the inner conductor (x1 < 0) the plasma field is 0; the analytic
 *      inside-star field still acts (Sec. 3.4.2).  Inside the outer conductor
 *      (x1 >= nr) particles fly ballistically (Sec. 3.4.2).
 *   R3 Time centring: x and E, B at step n, u at n-1/2; B is stored at integer
 *      time and advanced by two half steps around the E update (Yee leapfrog,
 *      Sec. 3.1 / Appendix A).
 *   R4 Azimuthal current: the charge crossing the meridional half-plane in one
 *      step is qw * dphi / (2 pi), dphi the azimuth swept by the straight 3-D
 *      move; it is shared over nodes with area (CIC) weights at the midpoint of
 *      the grid-coordinate path.
 *   R5 Deposited quantity: F = charge crossing each dual face during the step
 *      (grid units); E^{n+1} = E^n + dt*c*curl(B) - F/dA.  The filter acts on F.
 *   R6 Filter: no remap at the radial ends; values beyond the ghost rows are lost.
 *   R7 Polar fold: the part of a 1-2-1 pass that lands beyond the axis is folded
 *      onto its mirror point, with + for the integer-j components (r, phi) and -
 *      for the half-integer-j component (th) (App. B).
 *   R8 Deletion: floor(x1) < -(n_filt+1) or floor(x1) >= nr + n_filt + 1.
 *   R9 Lossy layer: sigma*(s), s = radial distance into the layer (in cells) at
 *      each component's own radial stagger; applied once per step to E^{n+1} and
 *      B^{n+1} after the full update (Sec. 3.4.1).
 *   R10 Injection: per surface cell j, sigma_j = mean of total E_r at (1/2, j) and
 *      (1/2, j+1); N_pp co-located pairs at rest at x1 = 1/2,
 *      x2 = j + (k+1/2)/N_pp, each of charge f_inj |sigma_j| dA_j / N_pp;
 *      none where |sigma_j| <= 1e-12 max_j |sigma_j| (zero up to rounding)
 *      (Sec. 5.3).
 *   R11 Spin-down luminosity (Sec. 5.3): the radial Poynting flux of the total
 *      field through the sphere of a node radius, with the staggered
 *      components averaged to the centres of the meridional cells on it.
 *   R12 Surface charge (Sec. 5.3): the jump of E_r across the conductor, i.e.
 *      the total E_r at (1/2, j) minus the analytic inside field's E_r at
 *      (r0, theta_j) (zero for the monopole fields); sigma_j averages j, j+1.
 *      Optional smoothing along theta: passes of (s_{j-1} + 2 s_j + s_{j+1})/4
 *      with each polar cell its own mirror image across the axis.
 *   R13 Variable-count injection, Eq. (volinjeq) as printed: n_j =
 *      f_inj |sigma_j| dA_j / q pairs of charge -+q, rounded stochastically
 *      (floor, plus one with probability equal to the fraction), the uniform
 *      number u = top 53 bits of SplitMix64 output (step * nth + j) + 1 of the
 *      stream seeded with inject_seed; at most pairs_per_cell pairs per cell
 *      (cells cut to it are counted); pair k of n_j at x2 = j + (k+1/2)/n_j.
 *      Ids as in R10: the counter advances by 2 * pairs_per_cell * nth.
 *   R14 Aligned dipole rotator fields (Sec. 4.3 dipole, Sec. 5.2 construction):
 *      B the dipole mu = B0 r0^3 everywhere; inside the star the corotation E;
 *      outside the vacuum field of the rotating conducting sphere with no net
 *      charge, E = -grad Phi, Phi = -(Omega mu r0^2 / 3 r^3)(3 cos^2 th - 1),
 *      which matches the inside potential's l = 2 part at r0.
 *   R15 Ties of the azimuth branch (adjudication, not arithmetic): a move that
 *      crosses the polar axis (X < 0, the displaced point's coordinate along
 *      the old cylindrical radius) sweeps the azimuth atan2(Y, X) (R4), whose
 *      sign is that of u_ph; the two signs differ by up to 2 pi.  When
 *      |u_ph| <= 2^-13 |u| that sign is set by the rounding of a nearly
 *      vanishing u_ph and both branches are valid.  Such ties are counted; a
 *      table of hints (step, id -> sign) from another run fixes the branch of
 *      the ties it lists, so a replay follows that run.  Without hints every
 *      tie keeps atan2's own branch.
 */
#include "picsar_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

enum { ORC_OK = 0, ORC_ECOURANT = -1, ORC_ERANGE = -2, ORC_ENOMEM = -3 };

struct orc_sim {
  orc_params p;
  int g;        /* ghost rows for fluxes and charge: n_filt + 2 */
  int ld;       /* row length nth + 1 */
  double dxi;   /* log map: ln(r_max/r_min)/nr; linear map: dr */
  double *f[6]; /* E_r, E_th, E_ph, B_r, B_th, B_ph : (nr+1) x (nth+1) */
  double *F[3]; /* F_r, F_th, F_ph with ghost rows : (nr+2g+1) x (nth+1) */
  int64_t np, cap;
  double *x1, *x2, *ur, *uth, *uph, *qw;
  int64_t *id;
  int64_t next_id;
  int64_t step;
  int64_t n_deleted, n_injected, n_capped;
  double *gq0; /* (G - Qbar) at the snapshot, (nr+1) x (nth+1) */
  int err;
  /* R15: ties met so far, and the hints (sorted by step, then id) */
  int64_t n_ties, nh;
  int64_t n_inject_ties; /* R13 draws within 1e-4 n_j of the rounding threshold */
  int64_t *h_step, *h_id;
  int *h_sign;
};

/* ------------------------------------------------------------------------- */
/* Stretching functions f_r, f_th and their inverses (Sec. 3.2).              */
/* log: xi = r0 ln(r/r0) uniform in x1; equal area: theta_A = -cos(theta)      */
/* uniform in x2 over [-1, 1].                                                 */
/* ------------------------------------------------------------------------- */
double orc_f_r(const orc_sim *s, double x1) {
  if (s->p.r_map == ORC_R_LOG) return s->p.r_min * exp(x1 * s->dxi);
  return s->p.r_min + x1 * s->dxi;
}
double orc_f_r_inv(const orc_sim *s, double r) {
  if (s->p.r_map == ORC_R_LOG) return log(r / s->p.r_min) / s->dxi;
  return (r - s->p.r_min) / s->dxi;
}
double orc_f_th(const orc_sim *s, double x2) {
  if (s->p.th_map == ORC_TH_EQUAL_AREA) return acos(1.0 - 2.0 * x2 / s->p.nth);
  return ORC_PI * x2 / s->p.nth;
}
double orc_f_th_inv(const orc_sim *s, double th) {
  if (s->p.th_map == ORC_TH_EQUAL_AREA) return 0.5 * s->p.nth * (1.0 - cos(th));
  return th * s->p.nth / ORC_PI;
}

/* Area and line elements, Eq. (linearea), Appendix A. */
static double dA_thph(double r, double ta, double tb) { return 2.0 * ORC_PI * r * r * (cos(ta) - cos(tb)); }
static double dA_rph(double ra, double rb, double th) { return ORC_PI * (rb * rb - ra * ra) * sin(th); }
static double dA_rth(double ra, double rb, double ta, double tb) { return 0.5 * (rb * rb - ra * ra) * (tb - ta); }
static double dL_r(double ra, double rb) { return rb - ra; }
static double dL_th(double r, double ta, double tb) { return r * (tb - ta); }
static double dL_ph(double r, double th) { return 2.0 * ORC_PI * r * sin(th); }

/* r_i = f_r(i), rb_i = f_r(i+1/2), th_j = f_th(j), tb_j = f_th(j+1/2): Eq. (rtdefs) */
static double R_(const orc_sim *s, int i) { return orc_f_r(s, (double)i); }
static double RB(const orc_sim *s, int i) { return orc_f_r(s, i + 0.5); }
static double T_(const orc_sim *s, int j) { return orc_f_th(s, (double)j); }
static double TB(const orc_sim *s, int j) { return orc_f_th(s, j + 0.5); }

/* Time step from a Courant number: dt = C * min over domain cells of
 * min(dr, r_inner * dtheta), c = 1 (Table 1 gives c in cells per step). */
double orc_courant_dt(const orc_params *p, double courant) {
  orc_sim tmp;
  memset(&tmp, 0, sizeof tmp);
  tmp.p = *p;
  tmp.dxi = (p->r_map == ORC_R_LOG) ? log(p->r_max / p->r_min) / p->nr : (p->r_max - p->r_min) / p->nr;
  double m = 1e300;
  for (int i = 0; i < p->nr; ++i) {
    double ra = orc_f_r(&tmp, i), rb = orc_f_r(&tmp, i + 1);
    for (int j = 0; j < p->nth; ++j) {
      double d = fmin(rb - ra, ra * (orc_f_th(&tmp, j + 1) - orc_f_th(&tmp, j)));
      if (d < m) m = d;
    }
  }
  return courant * m;
}

/* ------------------------------------------------------------------------- */
/* storage helpers                                                           */
/* ------------------------------------------------------------------------- */
#define FI(s, i, j) ((size_t)(i) * (size_t)(s)->ld + (size_t)(j))
#define GI(s, i, j) ((size_t)((i) + (s)->g) * (size_t)(s)->ld + (size_t)(j))

static size_t field_size(const orc_sim *s) { return (size_t)(s->p.nr + 1) * s->ld; }
static size_t ghost_size(const orc_sim *s) { return (size_t)(s->p.nr + 2 * s->g + 1) * s->ld; }

orc_sim *orc_create(const orc_params *p) {
  orc_sim *s = (orc_sim *)calloc(1, sizeof *s);
  if (!s) return NULL;
  s->p = *p;
  if (s->p.q_over_m == 0.0) s->p.q_over_m = 1.0;
  s->g = p->n_filt + 2;
  s->ld = p->nth + 1;
  s->dxi = (p->r_map == ORC_R_LOG) ? log(p->r_max / p->r_min) / p->nr : (p->r_max - p->r_min) / p->nr;
  for (int c = 0; c < 6; ++c) s->f[c] = (double *)calloc(field_size(s), sizeof(double));
  for (int c = 0; c < 3; ++c) s->F[c] = (double *)calloc(ghost_size(s), sizeof(double));
  return s;
}

void orc_destroy(orc_sim *s) {
  if (!s) return;
  for (int c = 0; c < 6; ++c) free(s->f[c]);
  for (int c = 0; c < 3; ++c) free(s->F[c]);
  free(s->x1); free(s->x2); free(s->ur); free(s->uth); free(s->uph); free(s->qw); free(s->id);
  free(s->gq0);
  free(s->h_step); free(s->h_id); free(s->h_sign);
  free(s);
}

int orc_last_error(const orc_sim *s) { return s->err; }
int32_t orc_ghost(const orc_sim *s) { return s->g; }

static void reserve(orc_sim *s, int64_t n) {
  if (n <= s->cap) return;
  int64_t c = s->cap ? s->cap : 1024;
  while (c < n) c *= 2;
  s->x1 = (double *)realloc(s->x1, c * sizeof(double));
  s->x2 = (double *)realloc(s->x2, c * sizeof(double));
  s->ur = (double *)realloc(s->ur, c * sizeof(double));
  s->uth = (double *)realloc(s->uth, c * sizeof(double));
  s->uph = (double *)realloc(s->uph, c * sizeof(double));
  s->qw = (double *)realloc(s->qw, c * sizeof(double));
  s->id = (int64_t *)realloc(s->id, c * sizeof(int64_t));
  s->cap = c;
}

void orc_load_particles(orc_sim *s, int64_t n, const double *x1, const double *x2,
                        const double *ur, const double *uth, const double *uph,
                        const double *qw, const int64_t *id) {
  reserve(s, s->np + n);
  for (int64_t k = 0; k < n; ++k) {
    int64_t d = s->np + k;
    s->x1[d] = x1[k]; s->x2[d] = x2[k];
    s->ur[d] = ur[k]; s->uth[d] = uth[k]; s->uph[d] = uph[k];
    s->qw[d] = qw[k];
    s->id[d] = id ? id[k] : s->next_id + k;
  }
  if (!id) s->next_id += n;
  else
    for (int64_t k = 0; k < n; ++k)
      if (id[k] + 1 > s->next_id) s->next_id = id[k] + 1;
  s->np += n;
}

int64_t orc_num_particles(const orc_sim *s) { return s->np; }

void orc_get_particles(const orc_sim *s, double *x1, double *x2, double *ur, double *uth,
                       double *uph, double *qw, int64_t *id) {
  for (int64_t k = 0; k < s->np; ++k) {
    if (x1) x1[k] = s->x1[k];
    if (x2) x2[k] = s->x2[k];
    if (ur) ur[k] = s->ur[k];
    if (uth) uth[k] = s->uth[k];
    if (uph) uph[k] = s->uph[k];
    if (qw) qw[k] = s->qw[k];
    if (id) id[k] = s->id[k];
  }
}

void orc_set_clock(orc_sim *s, int64_t step, int64_t next_id) {
  s->step = step;
  s->next_id = next_id;
}
int64_t orc_get_step(const orc_sim *s) { return s->step; }

void orc_get_fields(const orc_sim *s, double *out6) {
  for (int c = 0; c < 6; ++c) memcpy(out6 + c * field_size(s), s->f[c], field_size(s) * sizeof(double));
}
static void vacuum_rt(const orc_sim *s, double r, double th, double t, int inside, double E[3], double B[3]);

/* Total field (Sec. 5.2: plasma plus the analytic field, by linearity) at
 * each component's staggered point, at the context's time step * dt; every
 * grid point is at r >= r0, where the outside analytic field applies. */
void orc_get_fields_total(const orc_sim *s, double *out6) {
  static const int SI[6] = {1, 0, 0, 0, 1, 1}, SJ[6] = {0, 1, 0, 1, 0, 1};
  const double t = s->step * s->p.dt;
  orc_get_fields(s, out6);
  for (int c = 0; c < 6; ++c) {
    const int imax = SI[c] ? s->p.nr - 1 : s->p.nr, jmax = SJ[c] ? s->p.nth - 1 : s->p.nth;
    for (int i = 0; i <= imax; ++i)
      for (int j = 0; j <= jmax; ++j) {
        double E[3], B[3];
        vacuum_rt(s, SI[c] ? RB(s, i) : orc_f_r(s, (double)i), SJ[c] ? TB(s, j) : T_(s, j), t, 0, E, B);
        out6[c * field_size(s) + FI(s, i, j)] += c < 3 ? E[c] : B[c - 3];
      }
  }
}
void orc_set_fields(orc_sim *s, const double *in6) {
  for (int c = 0; c < 6; ++c) memcpy(s->f[c], in6 + c * field_size(s), field_size(s) * sizeof(double));
}
void orc_get_flux(const orc_sim *s, double *out3) {
  for (int c = 0; c < 3; ++c) memcpy(out3 + c * ghost_size(s), s->F[c], ghost_size(s) * sizeof(double));
}

void orc_counters(const orc_sim *s, int64_t *out5) {
  out5[0] = s->np;
  out5[1] = s->n_deleted;
  out5[2] = s->n_injected;
  out5[3] = s->next_id;
  out5[4] = s->n_capped;
}

/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the state advances by the
 * golden-ratio increment and each output is the state through the variant-13
 * mixing function; output n + 1 of the stream seeded with `seed` is therefore
 * the mix of seed + (n + 1) * increment. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* ------------------------------------------------------------------------- */
/* Analytic "initial" (vacuum) fields, Sec. 5.2 Eqs. (initialfields_outside)  */
/* and (initialfields_inside); the dipole + corotation field of Sec. 4.3; and  */
/* a uniform B_z used by the single-particle tests.  Spin-up: Omega rises      */
/* linearly to its final value over t_spin (Sec. 5.2); R_l = c / Omega_final.  */
/* ------------------------------------------------------------------------- */
static double omega_at(const orc_sim *s, double t) {
  if (s->p.t_spin > 0.0 && t < s->p.t_spin) return s->p.omega * (t / s->p.t_spin);
  return s->p.omega;
}

static void vacuum_rt(const orc_sim *s, double r, double th, double t, int inside, double E[3], double B[3]) {
  const double r0 = s->p.r_min, b0 = s->p.b0, st = sin(th), ct = cos(th);
  const double W = omega_at(s, t); /* Omega(t)/c with c = 1 */
  E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = 0.0;
  switch (s->p.vacuum) {
    case ORC_VAC_MONOPOLE:
      B[0] = b0 * (r0 / r) * (r0 / r);
      break;
    case ORC_VAC_MONOPOLE_ROTATOR:
      B[0] = b0 * (r0 / r) * (r0 / r);
      if (!inside) {
        double a = b0 * r0 * r0 * r0 * r0 / (r * r * r) * W; /* B0 r0^4 / (r^3 R_l) */
        E[0] = -2.0 * a * ct;
        E[1] = -a * st;
      } else {
        E[1] = -b0 * r0 * r0 / r * W * st; /* B0 r0^2 / (r R_l) */
      }
      break;
    case ORC_VAC_UNIFORM_BZ:
      B[0] = b0 * ct;
      B[1] = -b0 * st;
      break;
    case ORC_VAC_DIPOLE_COROT: {
      double mu = b0 * r0 * r0 * r0;
      B[0] = 2.0 * mu * ct / (r * r * r);
      B[1] = mu * st / (r * r * r);
      E[0] = mu * W * st * st / (r * r);
      E[1] = -mu * W * 2.0 * st * ct / (r * r);
      break;
    }
    case ORC_VAC_DIPOLE_ROTATOR: { /* reading R14 */
      double mu = b0 * r0 * r0 * r0;
      B[0] = 2.0 * mu * ct / (r * r * r);
      B[1] = mu * st / (r * r * r);
      if (inside) { /* corotation: -(Omega x r) x B */
        E[0] = mu * W * st * st / (r * r);
        E[1] = -mu * W * 2.0 * st * ct / (r * r);
      } else { /* -grad of -(Omega mu r0^2 / 3 r^3)(3 cos^2 - 1) */
        double a = mu * W * r0 * r0 / (r * r * r * r);
        E[0] = -a * (3.0 * ct * ct - 1.0);
        E[1] = -a * 2.0 * st * ct;
      }
      break;
    }
    default:
      break;
  }
}

void orc_vacuum_fields(const orc_sim *s, double x1, double x2, double t, double E[3], double B[3]) {
  vacuum_rt(s, orc_f_r(s, x1), orc_f_th(s, x2), t, x1 < 0.0, E, B);
}

/* ------------------------------------------------------------------------- */
/* Field gather (reading R2).  Staggering of Eq. (offseteq):                  */
/*   E_r (i+1/2, j)  E_th (i, j+1/2)  E_ph (i, j)                              */
/*   B_r (i, j+1/2)  B_th (i+1/2, j)  B_ph (i+1/2, j+1/2)                       */
/* ------------------------------------------------------------------------- */
static const int STAG_I[6] = {1, 0, 0, 0, 1, 1}; /* 1: half-integer radial position */
static const int STAG_J[6] = {0, 1, 0, 1, 0, 1}; /* 1: half-integer meridional position */
static const int AXIS_PARITY[6] = {1, -1, -1, 1, -1, -1};

static double comp_at(const orc_sim *s, int c, int i, int j) {
  const int nr = s->p.nr, nt = s->p.nth;
  const int imax = STAG_I[c] ? nr - 1 : nr;
  if (i < 0 || i > imax) return 0.0; /* conductor interior */
  if (STAG_J[c]) {
    if (j == -1) return AXIS_PARITY[c] * s->f[c][FI(s, i, 0)];
    if (j == nt) return AXIS_PARITY[c] * s->f[c][FI(s, i, nt - 1)];
    if (j < -1 || j > nt) return 0.0;
  } else if (j < 0 || j > nt) {
    return 0.0;
  }
  return s->f[c][FI(s, i, j)];
}

static double interp(const orc_sim *s, int c, double x1, double x2) {
  double p1 = x1 - 0.5 * STAG_I[c], p2 = x2 - 0.5 * STAG_J[c];
  double fi = floor(p1), fj = floor(p2);
  int i0 = (int)fi, j0 = (int)fj;
  double w1 = p1 - fi, w2 = p2 - fj;
  return (1 - w1) * (1 - w2) * comp_at(s, c, i0, j0) + w1 * (1 - w2) * comp_at(s, c, i0 + 1, j0) +
         (1 - w1) * w2 * comp_at(s, c, i0, j0 + 1) + w1 * w2 * comp_at(s, c, i0 + 1, j0 + 1);
}

/* Total field at a particle = plasma field on the grid + analytic field
 * (Sec. 5.2: "the total field is simply the sum"). */
void orc_gather(const orc_sim *s, double x1, double x2, double t, double E[3], double B[3]) {
  orc_vacuum_fields(s, x1, x2, t, E, B);
  if (x1 < 0.0 || x1 >= s->p.nr) return; /* no plasma field inside the conductors */
  for (int c = 0; c < 3; ++c) E[c] += interp(s, c, x1, x2);
  for (int c = 0; c < 3; ++c) B[c] += interp(s, 3 + c, x1, x2);
}

/* ------------------------------------------------------------------------- */
/* Relativistic pushers (Sec. 2), Cartesian components, c = 1.               */
/* qmdt = (q/m) dt of the particle; u = gamma v is updated in place.          */
/* ------------------------------------------------------------------------- */
static void cross(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Boris (1970): half electric kick, magnetic rotation through the tangent
 * vector t = (qdt/2m) B / gamma, second half electric kick. */
static void push_boris(double qmdt, const double E[3], const double B[3], double u[3]) {
  double h = 0.5 * qmdt, um[3], t[3], sv[3], up[3], c1[3], c2[3];
  for (int k = 0; k < 3; ++k) um[k] = u[k] + h * E[k];
  double g = sqrt(1.0 + dot(um, um));
  for (int k = 0; k < 3; ++k) t[k] = h * B[k] / g;
  double tt = dot(t, t);
  for (int k = 0; k < 3; ++k) sv[k] = 2.0 * t[k] / (1.0 + tt);
  cross(um, t, c1);
  for (int k = 0; k < 3; ++k) up[k] = um[k] + c1[k];
  cross(up, sv, c2);
  for (int k = 0; k < 3; ++k) u[k] = um[k] + c2[k] + h * E[k];
}

/* Vay (2008): the magnetic half step of the second half uses the new
 * velocity, u_new = u' + (u_new/gamma_new) x tau with
 * u' = u + qdt/m (E + v/2 x B) and tau = (qdt/2m) B; gamma_new solves the
 * quadratic in gamma^2 that follows from |u_new|^2 = gamma_new^2 - 1. */
static void push_vay(double qmdt, const double E[3], const double B[3], double u[3]) {
  double g0 = sqrt(1.0 + dot(u, u)), v[3], tau[3], vxt[3], up[3], t[3], uxt[3];
  for (int k = 0; k < 3; ++k) { v[k] = u[k] / g0; tau[k] = 0.5 * qmdt * B[k]; }
  cross(v, tau, vxt);
  for (int k = 0; k < 3; ++k) up[k] = u[k] + qmdt * E[k] + vxt[k];
  double tau2 = dot(tau, tau), ustar = dot(up, tau);
  double sigma = 1.0 + dot(up, up) - tau2;
  double g = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (tau2 + ustar * ustar))));
  for (int k = 0; k < 3; ++k) t[k] = tau[k] / g;
  double sfac = 1.0 / (1.0 + dot(t, t)), ut = dot(up, t);
  cross(up, t, uxt);
  for (int k = 0; k < 3; ++k) u[k] = sfac * (up[k] + ut * t[k] + uxt[k]);
}

void orc_push(int32_t pusher, double qmdt, const double E[3], const double B[3], double u[3]) {
  if (pusher == ORC_BORIS) push_boris(qmdt, E, B, u);
  else push_vay(qmdt, E, B, u);
}

/* ------------------------------------------------------------------------- */
/* Villasenor-Buneman deposit (Eq. Jcons, Sec. 3.3) in grid coordinates.      */
/* The particle is a unit square in grid coordinates.  For a straight path    */
/* p -> q that stays in cell (ic, jc), the charge crossing each dual face is   */
/* the time integral of q v times the overlap of the square with that face:    */
/*   F_r(ic+1/2, jc)   += qw dx1 (1 - m2)     F_r(ic+1/2, jc+1) += qw dx1 m2     */
/*   F_th(ic, jc+1/2)  += qw dx2 (1 - m1)     F_th(ic+1, jc+1/2) += qw dx2 m1    */
/* with m the path midpoint in the cell's local coordinates.  A path that      */
/* crosses grid lines is split where it crosses them.                          */
/* ------------------------------------------------------------------------- */
static int cell_j(const orc_sim *s, double x2) {
  int j = (int)floor(x2);
  if (j > s->p.nth - 1) j = s->p.nth - 1;
  if (j < 0) j = 0;
  return j;
}

static int add_ghost(orc_sim *s, double *a, int i, int j, double v) {
  if (i < -s->g || i > s->p.nr + s->g || j < 0 || j > s->p.nth) {
    if (v != 0.0) { s->err = ORC_ERANGE; return -1; }
    return 0;
  }
  a[GI(s, i, j)] += v;
  return 0;
}

static void vb_segment(orc_sim *s, double *fr, double *fth, double qw, int ic, int jc,
                       double p1, double p2, double q1, double q2) {
  double d1 = q1 - p1, d2 = q2 - p2;
  double m1 = 0.5 * (p1 + q1) - ic, m2 = 0.5 * (p2 + q2) - jc;
  add_ghost(s, fr, ic, jc, qw * d1 * (1.0 - m2));
  add_ghost(s, fr, ic, jc + 1, qw * d1 * m2);
  add_ghost(s, fth, ic, jc, qw * d2 * (1.0 - m1));
  add_ghost(s, fth, ic + 1, jc, qw * d2 * m1);
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int vb_path(orc_sim *s, double *fr, double *fth, double qw, double a1, double a2, double b1, double b2) {
  int ia = (int)floor(a1), ib = (int)floor(b1), ja = cell_j(s, a2), jb = cell_j(s, b2);
  if (abs(ib - ia) > 1 || abs(jb - ja) > 1) { s->err = ORC_ECOURANT; return -1; }
  /* crossing parameters along the path (0..1) */
  double sx = 2.0, sy = 2.0;
  if (ib != ia) sx = ((ia > ib ? ia : ib) - a1) / (b1 - a1);
  if (jb != ja) sy = ((ja > jb ? ja : jb) - a2) / (b2 - a2);
  double P1 = a1, P2 = a2;
  int ic = ia, jc = ja;
  for (int ev = 0; ev < 2; ++ev) {
    int xfirst = sx <= sy;
    double sn = xfirst ? sx : sy;
    if (sn > 1.0) break;
    double Q1, Q2;
    if (xfirst) {
      Q1 = (ia > ib ? ia : ib);
      Q2 = clampd(a2 + sn * (b2 - a2), jc, jc + 1);
    } else {
      Q2 = (ja > jb ? ja : jb);
      Q1 = clampd(a1 + sn * (b1 - a1), ic, ic + 1);
    }
    vb_segment(s, fr, fth, qw, ic, jc, P1, P2, Q1, Q2);
    P1 = Q1; P2 = Q2;
    if (xfirst) { ic = ib; sx = 2.0; } else { jc = jb; sy = 2.0; }
  }
  vb_segment(s, fr, fth, qw, ic, jc, P1, P2, b1, b2);
  return 0;
}

int orc_deposit_path(const orc_sim *s, double qw, double a1, double a2, double b1, double b2,
                     double *fr, double *fth) {
  orc_sim *m = (orc_sim *)s; /* only the error word is touched */
  int e0 = m->err;
  int r = vb_path(m, fr, fth, qw, a1, a2, b1, b2);
  m->err = e0;
  return r;
}

/* area (CIC) weights of the unit-square shape over the four nearest nodes */
static void cic_add(orc_sim *s, double *a, double x1, double x2, double v) {
  double fi = floor(x1), fj = floor(x2);
  int i0 = (int)fi, j0 = (int)fj;
  double w1 = x1 - fi, w2 = x2 - fj;
  add_ghost(s, a, i0, j0, v * (1 - w1) * (1 - w2));
  add_ghost(s, a, i0 + 1, j0, v * w1 * (1 - w2));
  add_ghost(s, a, i0, j0 + 1, v * (1 - w1) * w2);
  add_ghost(s, a, i0 + 1, j0 + 1, v * w1 * w2);
}

/* ------------------------------------------------------------------------- */
/* 1-2-1 digital filter, Eq. (filtereq), with the polar remapping of App. B    */
/* (reading R7) and no remap at the radial ends (reading R6).                  */
/* half_j = 1 for arrays at half-integer j (F_th); sign = fold sign.           */
/* ------------------------------------------------------------------------- */
void orc_filter_pass(const orc_sim *s, double *f, int32_t half_j, int32_t sign) {
  const int rows = s->p.nr + 2 * s->g + 1, ld = s->ld, nt = s->p.nth;
  const int nj = half_j ? nt : nt + 1; /* valid entries per row */
  double *tmp = (double *)calloc((size_t)rows * ld, sizeof(double));
  /* meridional pass */
  for (int r = 0; r < rows; ++r) {
    const double *in = f + (size_t)r * ld;
    double *out = tmp + (size_t)r * ld;
    for (int j = 0; j < nj; ++j) {
      double v = 0.5 * in[j];
      if (j - 1 >= 0) v += 0.25 * in[j - 1];
      if (j + 1 < nj) v += 0.25 * in[j + 1];
      out[j] = v;
    }
    /* what the pass would put beyond the axis is folded onto the mirror point */
    double north = 0.25 * in[0], south = 0.25 * in[nj - 1];
    if (half_j) { /* mirror of j = -1/2 is +1/2; of nt+1/2 is nt-1/2 */
      out[0] += sign * north;
      out[nj - 1] += sign * south;
    } else {      /* axis nodes j = 0, nt; mirror of -1 is 1, of nt+1 is nt-1 */
      out[1] += sign * north;
      out[nt - 1] += sign * south;
    }
  }
  /* radial pass */
  for (int r = 0; r < rows; ++r)
    for (int j = 0; j < nj; ++j) {
      double v = 0.5 * tmp[(size_t)r * ld + j];
      if (r - 1 >= 0) v += 0.25 * tmp[(size_t)(r - 1) * ld + j];
      if (r + 1 < rows) v += 0.25 * tmp[(size_t)(r + 1) * ld + j];
      f[(size_t)r * ld + j] = v;
    }
  free(tmp);
}

/* ------------------------------------------------------------------------- */
/* Field solve, Appendix A, Eqs. (discreteeq), (erpolarupdate), with the       */
/* conducting radial boundaries of Sec. 3.4.1 (E_th = E_ph = 0 at i = 0, nr,   */
/* never updated; B_r there changes only through E_ph, which is held at 0) and */
/* B_th = E_ph = 0 on the axis.                                               */
/* ------------------------------------------------------------------------- */
static void b_update(orc_sim *s, double h) {
  const int nr = s->p.nr, nt = s->p.nth;
  double *Er = s->f[0], *Et = s->f[1], *Ep = s->f[2], *Br = s->f[3], *Bt = s->f[4], *Bp = s->f[5];
  for (int i = 0; i <= nr; ++i)
    for (int j = 0; j < nt; ++j) {
      double ri = R_(s, i);
      double rhs = Ep[FI(s, i, j)] * dL_ph(ri, T_(s, j)) - Ep[FI(s, i, j + 1)] * dL_ph(ri, T_(s, j + 1));
      Br[FI(s, i, j)] += h * rhs / dA_thph(ri, T_(s, j), T_(s, j + 1));
    }
  for (int i = 0; i < nr; ++i)
    for (int j = 1; j < nt; ++j) {
      double tj = T_(s, j);
      double rhs = Ep[FI(s, i + 1, j)] * dL_ph(R_(s, i + 1), tj) - Ep[FI(s, i, j)] * dL_ph(R_(s, i), tj);
      Bt[FI(s, i, j)] += h * rhs / dA_rph(R_(s, i), R_(s, i + 1), tj);
    }
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nt; ++j) {
      double ra = R_(s, i), rb = R_(s, i + 1), ta = T_(s, j), tb = T_(s, j + 1);
      double rhs = (Et[FI(s, i, j)] * dL_th(ra, ta, tb) - Et[FI(s, i + 1, j)] * dL_th(rb, ta, tb)) -
                   (Er[FI(s, i, j)] * dL_r(ra, rb) - Er[FI(s, i, j + 1)] * dL_r(ra, rb));
      Bp[FI(s, i, j)] += h * rhs / dA_rth(ra, rb, ta, tb);
    }
}

static void e_update(orc_sim *s, double dt, int with_current) {
  const int nr = s->p.nr, nt = s->p.nth;
  double *Er = s->f[0], *Et = s->f[1], *Ep = s->f[2], *Br = s->f[3], *Bt = s->f[4], *Bp = s->f[5];
  double *Fr = s->F[0], *Ft = s->F[1], *Fp = s->F[2];
  /* E_r at (i+1/2, j), the polar caps j = 0 and j = nt by Eq. (erpolarupdate) */
  for (int i = 0; i < nr; ++i) {
    double rb = RB(s, i);
    for (int j = 0; j <= nt; ++j) {
      double circ, area;
      if (j == 0) {
        circ = Bp[FI(s, i, 0)] * dL_ph(rb, TB(s, 0));
        area = dA_thph(rb, 0.0, TB(s, 0));
      } else if (j == nt) {
        circ = -Bp[FI(s, i, nt - 1)] * dL_ph(rb, TB(s, nt - 1));
        area = dA_thph(rb, TB(s, nt - 1), ORC_PI);
      } else {
        circ = Bp[FI(s, i, j)] * dL_ph(rb, TB(s, j)) - Bp[FI(s, i, j - 1)] * dL_ph(rb, TB(s, j - 1));
        area = dA_thph(rb, TB(s, j - 1), TB(s, j));
      }
      double src = with_current ? Fr[GI(s, i, j)] : 0.0;
      Er[FI(s, i, j)] += (dt * circ - src) / area;
    }
  }
  /* E_th at (i, j+1/2), interior radii only */
  for (int i = 1; i < nr; ++i)
    for (int j = 0; j < nt; ++j) {
      double tb = TB(s, j), ra = RB(s, i - 1), rb = RB(s, i);
      double circ = Bp[FI(s, i - 1, j)] * dL_ph(ra, tb) - Bp[FI(s, i, j)] * dL_ph(rb, tb);
      double src = with_current ? Ft[GI(s, i, j)] : 0.0;
      Et[FI(s, i, j)] += (dt * circ - src) / dA_rph(ra, rb, tb);
    }
  /* E_ph at (i, j), interior radii and off the axis */
  for (int i = 1; i < nr; ++i)
    for (int j = 1; j < nt; ++j) {
      double ra = RB(s, i - 1), rb = RB(s, i), ta = TB(s, j - 1), tb = TB(s, j);
      double circ = (Bt[FI(s, i, j)] * dL_th(rb, ta, tb) - Bt[FI(s, i - 1, j)] * dL_th(ra, ta, tb)) -
                    (Br[FI(s, i, j)] * dL_r(ra, rb) - Br[FI(s, i, j - 1)] * dL_r(ra, rb));
      double src = with_current ? Fp[GI(s, i, j)] : 0.0;
      Ep[FI(s, i, j)] += (dt * circ - src) / dA_rth(ra, rb, ta, tb);
    }
}

/* Lossy layer, Eq. (EBcond): field <- (1 - sigma*) field inside the outer
 * absorb_cells cells, sigma* rising from 0 at the inner edge (reading R9). */
static double sigma_star(const orc_sim *s, double rho) {
  const int L = s->p.absorb_cells;
  if (s->p.absorb_profile == ORC_ABSORB_NONE || L <= 0) return 0.0;
  double x = rho - (s->p.nr - L);
  if (x <= 0.0) return 0.0;
  double u = x / L;
  if (s->p.absorb_profile == ORC_ABSORB_QUADRATIC) {
    double smax = s->p.absorb_sigma_max > 0 ? s->p.absorb_sigma_max : 3.0 / L;
    return smax * u * u;
  }
  double smax = s->p.absorb_sigma_max > 0 ? s->p.absorb_sigma_max : 2.0 / L;
  return smax * u;
}

static void lossy(orc_sim *s) {
  if (s->p.absorb_profile == ORC_ABSORB_NONE || s->p.absorb_cells <= 0) return;
  for (int c = 0; c < 6; ++c)
    for (int i = 0; i <= s->p.nr; ++i) {
      double k = 1.0 - sigma_star(s, i + 0.5 * STAG_I[c]);
      if (k == 1.0) continue;
      for (int j = 0; j <= s->p.nth; ++j) s->f[c][FI(s, i, j)] *= k;
    }
}

/* one leapfrog: B half step, E full step, B half step (reading R3) */
static void field_solve(orc_sim *s, int with_current) {
  b_update(s, 0.5 * s->p.dt);
  e_update(s, s->p.dt, with_current);
  b_update(s, 0.5 * s->p.dt);
  lossy(s);
}

void orc_field_step(orc_sim *s, int32_t nsteps) {
  for (int n = 0; n < nsteps; ++n) {
    field_solve(s, 0);
    s->step += 1;
  }
}

/* ------------------------------------------------------------------------- */
/* Particle step: gather, push, move, deposit, boundary decision             */
/* (Secs. 2, 3.3, 3.4.2).  The push and move run in Cartesian components of   */
/* the meridional plane phi = 0; after the move the particle is rotated back  */
/* to phi = 0 (axisymmetry), which also reflects it through the polar axis.   */
/* ------------------------------------------------------------------------- */
/* R15: the hinted branch of a tie at (current step, id), else phi's own */
static double tie_branch(orc_sim *s, int64_t id, double phi) {
  int sg = phi < 0 ? -1 : 1;
  s->n_ties++;
  for (int64_t lo = 0, hi = s->nh; lo < hi;) {
    int64_t mid = (lo + hi) / 2;
    if (s->h_step[mid] == s->step && s->h_id[mid] == id) { sg = s->h_sign[mid] < 0 ? -1 : 1; break; }
    if (s->h_step[mid] < s->step || (s->h_step[mid] == s->step && s->h_id[mid] < id)) lo = mid + 1;
    else hi = mid;
  }
  return sg * fabs(phi);
}

static void particle_step(orc_sim *s, int64_t k, double t, int *del) {
  const int nr = s->p.nr;
  double x1 = s->x1[k], x2 = s->x2[k], qw = s->qw[k];
  double r = orc_f_r(s, x1), th = orc_f_th(s, x2), st = sin(th), ct = cos(th);
  /* local spherical basis at phi = 0 in Cartesian (x = R, y = phi, z) */
  double u[3] = {s->ur[k] * st + s->uth[k] * ct, s->uph[k], s->ur[k] * ct - s->uth[k] * st};
  if (x1 < nr) { /* ballistic inside the outer conductor */
    double Es[3], Bs[3], E[3], B[3];
    orc_gather(s, x1, x2, t, Es, Bs);
    E[0] = Es[0] * st + Es[1] * ct; E[1] = Es[2]; E[2] = Es[0] * ct - Es[1] * st;
    B[0] = Bs[0] * st + Bs[1] * ct; B[1] = Bs[2]; B[2] = Bs[0] * ct - Bs[1] * st;
    double qmdt = (qw > 0 ? 1.0 : -1.0) * s->p.q_over_m * s->p.dt;
    orc_push(s->p.pusher, qmdt, E, B, u);
  }
  double g = sqrt(1.0 + dot(u, u));
  double X = r * st + u[0] / g * s->p.dt, Y = u[1] / g * s->p.dt, Z = r * ct + u[2] / g * s->p.dt;
  double R = hypot(X, Y), phi = atan2(Y, X), rn = hypot(R, Z), thn = atan2(R, Z);
  if (X < 0 && u[1] * u[1] <= dot(u, u) / (8192.0 * 8192.0)) phi = tie_branch(s, s->id[k], phi); /* R15 */
  double cp = R > 0 ? X / R : 1.0, sp = R > 0 ? Y / R : 0.0;
  double ux = cp * u[0] + sp * u[1], uy = -sp * u[0] + cp * u[1], uz = u[2];
  double stn = rn > 0 ? R / rn : 0.0, ctn = rn > 0 ? Z / rn : 1.0;
  double nx1 = orc_f_r_inv(s, rn), nx2 = orc_f_th_inv(s, thn);
  nx2 = clampd(nx2, 0.0, (double)s->p.nth);
  /* Villasenor-Buneman along the grid-coordinate path, and the azimuthal flux */
  vb_path(s, s->F[0], s->F[1], qw, x1, x2, nx1, nx2);
  cic_add(s, s->F[2], 0.5 * (x1 + nx1), 0.5 * (x2 + nx2), qw * phi / (2.0 * ORC_PI));
  s->x1[k] = nx1; s->x2[k] = nx2;
  s->ur[k] = ux * stn + uz * ctn;
  s->uth[k] = ux * ctn - uz * stn;
  s->uph[k] = uy;
  int ci = (int)floor(nx1);
  *del = ci < -(s->p.n_filt + 1) || ci >= nr + s->p.n_filt + 1;
}

/* Surface injection, Sec. 5.3 Eq. (volinjeq), readings R10, R12, R13. */
static void inject(orc_sim *s, double t) {
  const int nt = s->p.nth, npp = s->p.pairs_per_cell;
  const double r0 = s->p.r_min, rb0 = RB(s, 0);
  double *sig = (double *)malloc(sizeof(double) * nt), *tmp = (double *)malloc(sizeof(double) * nt);
  double smax = 0.0;
  reserve(s, s->np + (int64_t)2 * npp * nt);
  for (int j = 0; j < nt; ++j) {
    double Ev[3], Bv[3], Ei[3], e0, e1;
    vacuum_rt(s, rb0, T_(s, j), t, 0, Ev, Bv);
    vacuum_rt(s, r0, T_(s, j), t, 1, Ei, Bv);
    e0 = (s->f[0][FI(s, 0, j)] + Ev[0]) - Ei[0];
    vacuum_rt(s, rb0, T_(s, j + 1), t, 0, Ev, Bv);
    vacuum_rt(s, r0, T_(s, j + 1), t, 1, Ei, Bv);
    e1 = (s->f[0][FI(s, 0, j + 1)] + Ev[0]) - Ei[0];
    sig[j] = 0.5 * (e0 + e1); /* jump of E_r across the surface */
  }
  for (int pass = 0; pass < s->p.inject_smooth; ++pass) {
    for (int j = 0; j < nt; ++j) {
      double a = sig[j > 0 ? j - 1 : 0], c = sig[j < nt - 1 ? j + 1 : nt - 1];
      tmp[j] = ((a + 2.0 * sig[j]) + c) * 0.25;
    }
    memcpy(sig, tmp, sizeof(double) * nt);
  }
  for (int j = 0; j < nt; ++j)
    if (fabs(sig[j]) > smax) smax = fabs(sig[j]);
  const uint64_t step = (uint64_t)s->step;
  for (int j = 0; j < nt; ++j) {
    double dA = 2.0 * ORC_PI * r0 * r0 * (cos(T_(s, j)) - cos(T_(s, j + 1)));
    int m;       /* pairs injected into cell j */
    double w;    /* |charge| of each */
    if (s->p.inject == ORC_INJECT_VARIABLE) {
      double x = s->p.f_inj * fabs(sig[j]) * dA / s->p.inject_q;
      w = s->p.inject_q;
      m = 0;
      if (fabs(sig[j]) > 1e-12 * smax && x > 0.0) {
        if (x >= npp + 1.0) {
          m = npp + 1;
        } else {
          double fl = floor(x);
          double u = (double)(orc_splitmix64(s->p.inject_seed, step * (uint64_t)nt + (uint64_t)j) >> 11) *
                     (1.0 / 9007199254740992.0);
          m = (int)fl + (u < x - fl ? 1 : 0);
          /* a near-tie: a relative change of 1e-4 in n_j (a surface field
           * held to a lower precision) could round this cell the other way */
          if (fabs(u - (x - fl)) <= 1e-4 * x) s->n_inject_ties++;
        }
        if (m > npp) { m = npp; s->n_capped++; }
      }
    } else {
      w = s->p.f_inj * fabs(sig[j]) * dA / npp;
      /* cells whose surface charge is zero up to rounding inject nothing */
      m = (fabs(sig[j]) > 1e-12 * smax && w > 0.0) ? npp : 0;
    }
    for (int k = 0; k < m; ++k)
      for (int sgn = 0; sgn < 2; ++sgn) {
        int64_t d = s->np++;
        s->x1[d] = 0.5;
        s->x2[d] = j + (k + 0.5) / m;
        s->ur[d] = s->uth[d] = s->uph[d] = 0.0;
        s->qw[d] = sgn == 0 ? w : -w;
        s->id[d] = s->next_id + ((int64_t)j * npp + k) * 2 + sgn;
        s->n_injected++;
      }
  }
  free(sig);
  free(tmp);
  s->next_id += (int64_t)2 * npp * nt;
}

/* Every particle's step with zeroed fluxes, then stable removal of those whose
 * shape left the domain. */
static void particles_pass(orc_sim *s, double t) {
  for (int c = 0; c < 3; ++c) memset(s->F[c], 0, ghost_size(s) * sizeof(double));
  int64_t w = 0;
  for (int64_t k = 0; k < s->np; ++k) {
    int del = 0;
    particle_step(s, k, t, &del);
    if (del) { s->n_deleted++; continue; }
    if (w != k) {
      s->x1[w] = s->x1[k]; s->x2[w] = s->x2[k];
      s->ur[w] = s->ur[k]; s->uth[w] = s->uth[k]; s->uph[w] = s->uph[k];
      s->qw[w] = s->qw[k]; s->id[w] = s->id[k];
    }
    ++w;
  }
  s->np = w;
}

/* The particle part of one step only, fields and clock left as they are: it
 * replays a sample of a large state without the full-grid field solve. */
void orc_particles_only(orc_sim *s) { particles_pass(s, s->step * s->p.dt); }

void orc_step(orc_sim *s, int32_t nsteps) {
  for (int n = 0; n < nsteps; ++n) {
    particles_pass(s, s->step * s->p.dt);
    for (int f = 0; f < s->p.n_filt; ++f) {
      orc_filter_pass(s, s->F[0], 0, +1);
      orc_filter_pass(s, s->F[1], 1, -1);
      orc_filter_pass(s, s->F[2], 0, +1);
    }
    field_solve(s, 1);
    s->step += 1;
    if (s->p.inject) inject(s, s->step * s->p.dt);
  }
}

/* ------------------------------------------------------------------------- */
/* Diagnostics                                                               */
/* ------------------------------------------------------------------------- */
/* Spin-down luminosity (Sec. 5.3, Fig. 7d): the radial Poynting flux
 * (E x B)_r (c = 1) of the total field, plasma plus analytic at time t,
 * through the sphere of each interior node radius r_i, 1 <= i <= nr - 1
 * (reading R11).  On the sphere, meridional cell j carries E_th(i, j+1/2);
 * B_ph, given at i -+ 1/2, is averaged to r_i; E_ph, given at the nodes j and
 * j+1, and B_th, at (i -+ 1/2, j) and (i -+ 1/2, j+1), are averaged to the
 * cell's centre; the analytic field is evaluated there.  Each cell adds
 * (E_th B_ph - E_ph B_th) 2 pi r_i^2 (cos th_j - cos th_{j+1}).  out[0] and
 * out[nr] are 0. */
void orc_luminosity(const orc_sim *s, double t, double *out) {
  const int nr = s->p.nr, nt = s->p.nth;
  for (int i = 0; i <= nr; ++i) out[i] = 0.0;
  for (int i = 1; i < nr; ++i) {
    const double r = orc_f_r(s, (double)i);
    double L = 0.0;
    for (int j = 0; j < nt; ++j) {
      double Ev[3], Bv[3];
      vacuum_rt(s, r, orc_f_th(s, j + 0.5), t, 0, Ev, Bv);
      const double et = s->f[1][FI(s, i, j)] + Ev[1];
      const double bp = 0.5 * (s->f[5][FI(s, i - 1, j)] + s->f[5][FI(s, i, j)]) + Bv[2];
      const double ep = 0.5 * (s->f[2][FI(s, i, j)] + s->f[2][FI(s, i, j + 1)]) + Ev[2];
      const double bt = 0.25 * (s->f[4][FI(s, i - 1, j)] + s->f[4][FI(s, i, j)] + s->f[4][FI(s, i - 1, j + 1)] +
                                s->f[4][FI(s, i, j + 1)]) + Bv[1];
      const double dA = 2.0 * ORC_PI * r * r * (cos(T_(s, j)) - cos(T_(s, j + 1)));
      L += (et * bp - ep * bt) * dA;
    }
    out[i] = L;
  }
}

void orc_node_charge(const orc_sim *s, int32_t absolute, double *q) {
  orc_sim *m = (orc_sim *)s;
  memset(q, 0, ghost_size(s) * sizeof(double));
  for (int64_t k = 0; k < s->np; ++k) cic_add(m, q, s->x1[k], s->x2[k], absolute ? fabs(s->qw[k]) : s->qw[k]);
}

/* Integral Gauss law per dual cell (reading R1): flux of E out of the dual
 * cell of node (i, j); polar caps close at the axis. */
static double gauss_G(const orc_sim *s, int i, int j) {
  const int nt = s->p.nth;
  double tlo = j > 0 ? TB(s, j - 1) : 0.0, thi = j < nt ? TB(s, j) : ORC_PI;
  double ra = RB(s, i - 1), rb = RB(s, i);
  double G = s->f[0][FI(s, i, j)] * dA_thph(rb, tlo, thi) - s->f[0][FI(s, i - 1, j)] * dA_thph(ra, tlo, thi);
  if (j < nt) G += s->f[1][FI(s, i, j)] * dA_rph(ra, rb, TB(s, j));
  if (j > 0) G -= s->f[1][FI(s, i, j - 1)] * dA_rph(ra, rb, TB(s, j - 1));
  return G;
}

static int gauss_imax(const orc_sim *s) {
  int L = s->p.absorb_profile == ORC_ABSORB_NONE ? 0 : s->p.absorb_cells;
  return s->p.nr - L - 1;
}

/* G - Qbar at interior nodes, Qbar = Q filtered like F_r (App. B: with a
 * filtered current the conserved charge is the filtered charge). */
static void gauss_diff(const orc_sim *s, double *out) {
  double *q = (double *)malloc(ghost_size(s) * sizeof(double));
  orc_node_charge(s, 0, q);
  for (int f = 0; f < s->p.n_filt; ++f) orc_filter_pass(s, q, 0, +1);
  memset(out, 0, field_size(s) * sizeof(double));
  for (int i = 1; i <= gauss_imax(s); ++i)
    for (int j = 0; j <= s->p.nth; ++j) out[FI(s, i, j)] = gauss_G(s, i, j) - q[GI(s, i, j)];
  free(q);
}

void orc_gauss_snapshot(orc_sim *s) {
  if (!s->gq0) s->gq0 = (double *)malloc(field_size(s) * sizeof(double));
  gauss_diff(s, s->gq0);
}

double orc_gauss_residual(const orc_sim *s) {
  double *d = (double *)malloc(field_size(s) * sizeof(double));
  double *qa = (double *)malloc(ghost_size(s) * sizeof(double));
  gauss_diff(s, d);
  orc_node_charge(s, 1, qa);
  double num = 0.0, den = 0.0;
  for (int i = 1; i <= gauss_imax(s); ++i)
    for (int j = 0; j <= s->p.nth; ++j) {
      double v = d[FI(s, i, j)] - (s->gq0 ? s->gq0[FI(s, i, j)] : 0.0);
      if (fabs(v) > num) num = fabs(v);
      if (qa[GI(s, i, j)] > den) den = qa[GI(s, i, j)];
    }
  free(d);
  free(qa);
  return den > 0 ? num / den : num;
}

/* Field energy 1/2 (E^2 + B^2) summed over the cells centred on each
 * component's staggered location (clipped to the domain). */
double orc_field_energy(const orc_sim *s) {
  double W = 0.0;
  for (int c = 0; c < 6; ++c) {
    int imax = STAG_I[c] ? s->p.nr - 1 : s->p.nr, jmax = STAG_J[c] ? s->p.nth - 1 : s->p.nth;
    for (int i = 0; i <= imax; ++i) {
      double a = i + 0.5 * STAG_I[c] - 0.5, b = a + 1.0;
      if (a < 0) a = 0;
      if (b > s->p.nr) b = s->p.nr;
      double ra = orc_f_r(s, a), rb = orc_f_r(s, b);
      for (int j = 0; j <= jmax; ++j) {
        double ta = j + 0.5 * STAG_J[c] - 0.5, tb = ta + 1.0;
        if (ta < 0) ta = 0;
        if (tb > s->p.nth) tb = s->p.nth;
        double vol = 2.0 * ORC_PI / 3.0 * (rb * rb * rb - ra * ra * ra) * (cos(orc_f_th(s, ta)) - cos(orc_f_th(s, tb)));
        double v = s->f[c][FI(s, i, j)];
        W += 0.5 * v * v * vol;
      }
    }
  }
  return W;
}

double orc_kinetic_energy(const orc_sim *s) {
  double K = 0.0;
  for (int64_t k = 0; k < s->np; ++k) {
    double u2 = s->ur[k] * s->ur[k] + s->uth[k] * s->uth[k] + s->uph[k] * s->uph[k];
    K += fabs(s->qw[k]) / s->p.q_over_m * (sqrt(1.0 + u2) - 1.0);
  }
  return K;
}

/* discrete div B: flux of B out of each primary cell (i, j), Eq. (maxti) */
void orc_divb(const orc_sim *s, double *out) {
  const int nr = s->p.nr, nt = s->p.nth;
  const double *Br = s->f[3], *Bt = s->f[4];
  for (int i = 0; i < nr; ++i)
    for (int j = 0; j < nt; ++j) {
      double ta = T_(s, j), tb = T_(s, j + 1), ra = R_(s, i), rb = R_(s, i + 1);
      out[(size_t)i * nt + j] = Br[FI(s, i + 1, j)] * dA_thph(rb, ta, tb) - Br[FI(s, i, j)] * dA_thph(ra, ta, tb) +
                                Bt[FI(s, i, j + 1)] * dA_rph(ra, rb, tb) - Bt[FI(s, i, j)] * dA_rph(ra, rb, ta);
    }
}

/* R15 hints: n entries (step, id, sign), any order; replaces the table */
static const int64_t *g_hs, *g_hi;
static int hint_cmp(const void *a, const void *b) {
  int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
  if (g_hs[i] != g_hs[j]) return g_hs[i] < g_hs[j] ? -1 : 1;
  if (g_hi[i] != g_hi[j]) return g_hi[i] < g_hi[j] ? -1 : 1;
  return 0;
}

void orc_set_axis_hints(orc_sim *s, int64_t n, const int64_t *steps, const int64_t *ids, const int32_t *signs) {
  free(s->h_step); free(s->h_id); free(s->h_sign);
  s->h_step = s->h_id = NULL;
  s->h_sign = NULL;
  s->nh = 0;
  if (n <= 0) return;
  int64_t *ord = (int64_t *)malloc(n * sizeof(int64_t));
  for (int64_t k = 0; k < n; ++k) ord[k] = k;
  g_hs = steps; g_hi = ids;
  qsort(ord, (size_t)n, sizeof(int64_t), hint_cmp);
  s->h_step = (int64_t *)malloc(n * sizeof(int64_t));
  s->h_id = (int64_t *)malloc(n * sizeof(int64_t));
  s->h_sign = (int *)malloc(n * sizeof(int));
  for (int64_t k = 0; k < n; ++k) {
    s->h_step[k] = steps[ord[k]];
    s->h_id[k] = ids[ord[k]];
    s->h_sign[k] = signs[ord[k]];
  }
  s->nh = n;
  free(ord);
}

int64_t orc_axis_ties(const orc_sim *s) { return s->n_ties; }

int64_t orc_inject_ties(const orc_sim *s) { return s->n_inject_ties; }

/*
 * picsar.h -- C-ABI of the GB300 (sm_103a) PICsar particle hot path.
 *
 * The library advances the 2.5D axisymmetric, relativistic, electromagnetic,
 * charge-conservative particle-in-cell method of Belyaev, "PICsar" (arXiv
 * 1407.1810) on its body-fitted, stretchable spherical (r, theta) grid:
 *   per step: field gather from the staggered Yee mesh (Eq. offseteq) plus the
 *   analytic "initial" field (Sec. 5.2); Vay or Boris push (Sec. 2) and the
 *   axisymmetric move (Sec. 3.3); the particle boundary rule (Sec. 3.4.2);
 *   Villasenor-Buneman charge-conserving deposit (Eq. Jcons, Sec. 3.3);
 *   N_filt passes of the 1-2-1 filter with the polar remap (App. B); the Yee
 *   field update in integral form (App. A, Eqs. discreteeq, erpolarupdate) with
 *   conducting radial boundaries and the lossy layer (Sec. 3.4.1, Eq. EBcond);
 *   surface pair injection (Sec. 5.3, Eq. volinjeq).
 *
 * Units: Lorentz-Heaviside with c = 1 (Sec. 2).  Grid: nr x nth cells, nodes
 * i = 0..nr (radial, i = 0 on the inner conductor r = r_min) and j = 0..nth
 * (j = 0 and j = nth on the polar axis).  A particle's grid coordinate is
 * (x1, x2) with r = f_r(x1), theta = f_th(x2) (Sec. 3.2).  Momentum is
 * u = gamma v in the local spherical basis (u_r, u_th, u_ph).  qw is the
 * signed macro-charge; the mass is |qw| / q_over_m.
 *
 * Conventions of every call:
 *   - the return value is PIC_OK (0) or a negative PIC_E* code; the message of
 *     the last failure on the calling thread is pic_last_error();
 *   - the library copies its inputs and never keeps a caller pointer;
 *   - outputs go to caller-owned buffers; a pointer argument marked "mem" is a
 *     host pointer when mem == PIC_MEM_HOST and a device pointer of the
 *     context's device when mem == PIC_MEM_DEVICE;
 *   - all GPU work runs on the stream given to pic_init_grid (a cudaStream_t,
 *     NULL = the legacy default stream).  pic_step enqueues its steps and
 *     synchronises the stream only at a particle sort (every sort_interval
 *     steps, to read the live count) or when it grows the particle buffer;
 *     calls that return data to the host synchronise that stream.
 * Errors found by a kernel (a particle moving more than one cell in a step, a
 * full particle buffer, a non-finite momentum) are latched in the context and
 * reported by the next call that synchronises.
 */
#ifndef PICSAR_H
#define PICSAR_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PIC_OK 0
#define PIC_EINVAL (-1)    /* bad argument or descriptor */
#define PIC_ENOMEM (-2)    /* device allocation failed */
#define PIC_ECUDA (-3)     /* a CUDA call failed */
#define PIC_ECAPACITY (-4) /* particle buffer full */
#define PIC_ENAN (-5)      /* non-finite particle momentum or position */
#define PIC_ECOURANT (-6)  /* a particle crossed more than one cell line in one step */
#define PIC_ETIMEOUT (-7)  /* a bounded device-side wait gave up */

/* enumerations */
enum { PIC_R_LINEAR = 0, PIC_R_LOG = 1 };                  /* f_r, Sec. 3.2 */
enum { PIC_TH_LINEAR = 0, PIC_TH_EQUAL_AREA = 1 };         /* f_th, Sec. 3.2 */
enum { PIC_ABSORB_NONE = 0, PIC_ABSORB_LINEAR = 1, PIC_ABSORB_QUADRATIC = 2 };
enum { PIC_VAC_NONE = 0, PIC_VAC_MONOPOLE = 1, PIC_VAC_MONOPOLE_ROTATOR = 2,
       PIC_VAC_UNIFORM_BZ = 3, PIC_VAC_DIPOLE_COROT = 4, PIC_VAC_DIPOLE_ROTATOR = 5 };
/* Surface injection (Sec. 5.3).  FIXED: pairs_per_cell pairs in every surface
 * cell, each of charge f_inj |sigma_j| dA_j / pairs_per_cell.  VARIABLE:
 * Eq. (volinjeq) as printed, n_j = f_inj |sigma_j| dA_j / inject_q pairs of
 * charge -+inject_q, rounded stochastically (floor, plus one with probability
 * equal to the fraction; the uniform number is the top 53 bits of SplitMix64
 * output step * nth + j + 1 of the stream seeded with inject_seed) and cut to
 * pairs_per_cell (cells cut are counted in pic_moments.inject_capped).  In
 * both modes sigma_j is the jump of E_r across the surface (total E_r at
 * (1/2, j) minus the analytic inside field's E_r at r0), averaged over j and
 * j+1, then smoothed by inject_smooth 1-2-1 passes along theta with each polar
 * cell its own mirror image; pair k of m in cell j sits at x1 = 1/2,
 * x2 = j + (k + 1/2)/m; ids advance by 2 pairs_per_cell nth every step. */
enum { PIC_INJECT_OFF = 0, PIC_INJECT_FIXED = 1, PIC_INJECT_VARIABLE = 2 };
enum { PIC_FP64 = 0, PIC_FP32 = 1 };
enum { PIC_VAY = 0, PIC_BORIS = 1 };
enum { PIC_MEM_HOST = 0, PIC_MEM_DEVICE = 1 };
enum { PIC_FIELDS_PLASMA = 0, PIC_FIELDS_TOTAL = 1 };

typedef struct pic_ctx pic_ctx;

/* Grid and physics of one simulation.  Zero-initialise, then set. */
typedef struct pic_desc {
  int32_t nr, nth;           /* cells in r and theta (>= 2 each) */
  double r_min, r_max;       /* inner (r0) and outer conductor radius, r_min > 0 */
  int32_t r_map, th_map;     /* PIC_R_*, PIC_TH_* stretching functions (Sec. 3.2) */
  double courant;            /* used when dt <= 0: dt = courant * min cell size */
  double dt;                 /* time step; > 0 overrides courant */
  int32_t n_filt;            /* 1-2-1 filter passes on the current (App. B), 0..16 */
  int32_t absorb_cells;      /* lossy layer width in cells (Sec. 3.4.1) */
  int32_t absorb_profile;    /* PIC_ABSORB_* */
  double absorb_sigma_max;   /* sigma* at the outer conductor; <= 0: 2/L linear, 3/L quadratic */
  int32_t vacuum;            /* PIC_VAC_* analytic field added at the particle (Sec. 5.2, 4.3);
                                DIPOLE_ROTATOR: dipole B (mu = b0 r0^3), corotation E inside,
                                outside the vacuum E of the rotating conductor with no net
                                charge, -grad of -(Omega mu r0^2 / 3 r^3)(3 cos^2 th - 1) */
  double b0;                 /* field strength at r0 */
  double omega;              /* final angular velocity of the star; R_l = c / omega */
  double t_spin;             /* linear spin-up time (Sec. 5.2); 0 = none */
  int32_t inject;            /* PIC_INJECT_*: surface pair injection each step (Sec. 5.3) */
  int32_t pairs_per_cell;    /* FIXED: pairs per surface cell per step; VARIABLE: the cap */
  double f_inj;              /* injection multiplier, 0 < f_inj <= 1 (Eq. volinjeq) */
  int32_t precision;         /* PIC_FP64 (plain FP64 path) or PIC_FP32 (cell+offset path) */
  int32_t pusher;            /* PIC_VAY or PIC_BORIS (Sec. 2) */
  double q_over_m;           /* |q|/m of both species; 0 means 1 */
  int32_t sort_interval;     /* FP32 path: steps between tile sorts (0 = 20);
                                FP64 path: steps between compactions */
  int64_t capacity;          /* particle slots to allocate (0 = 2x the first load + injection room) */
  double flux_quantum;       /* FP32 path: least charge of one fixed-point flux unit; 0 = automatic.
                                The unit is 2^(e - 36), e = ceil(log2 max |qw|) over every charge
                                the context has held (loaded or injected, raised on the device),
                                and at least this value rounded up to a power of two. */
  int32_t tile_shape;        /* FP32 path: tile of the shared-memory deposit, 0 = 16x16 cells,
                                1 = 8 (r) x 32 (theta), 2 = 32 x 8 */
  int32_t inject_smooth;     /* 1-2-1 passes over sigma_j along theta, 0..64 */
  double inject_q;           /* VARIABLE injection: |charge| of each injected particle, > 0 */
  uint64_t inject_seed;      /* VARIABLE injection: seed of the stochastic rounding */
} pic_desc;

/* Diagnostics returned by pic_get_moments. */
typedef struct pic_moments {
  int64_t live;              /* live particles */
  int64_t deleted;           /* particles removed at the conductors so far */
  int64_t injected;          /* particles injected so far */
  int64_t step;              /* steps taken */
  double time;               /* step * dt */
  double dt;                 /* time step in use */
  double kinetic_energy;     /* sum |qw|/q_over_m (gamma - 1) */
  double field_energy;       /* 1/2 sum (E^2 + B^2) dV of the plasma field */
  double gauss_residual;     /* max |(G - Qbar) - (G - Qbar)_0| / max sum |qw| CIC over the
                                interior nodes 1 <= i <= nr - absorb_cells - 1 (App. B, Sec. 2) */
  double total_charge;       /* sum qw */
  int64_t inject_capped;     /* VARIABLE injection: cell-steps whose count was cut to pairs_per_cell */
  int64_t axis_ties;         /* axis crossings whose azimuth branch was a tie (see pic_get_axis_ties) */
} pic_moments;

/* Create a context: allocates the grid arrays on the current CUDA device and
 * uploads the metric tables.  d: descriptor (copied).  stream: cudaStream_t or
 * NULL.  *out receives the handle.  Errors: PIC_EINVAL (bad descriptor),
 * PIC_ENOMEM, PIC_ECUDA. */
int pic_init_grid(pic_ctx **out, const pic_desc *d, void *stream);

/* Append n particles (Sec. 3.3 state).  x1, x2: grid coordinates; u_r, u_th,
 * u_ph: gamma v in the local spherical basis; qw: signed macro-charge (nonzero).
 * All arrays are FP64 of length n, host or device per mem; page-locked
 * (pinned) host arrays are read in place by the GPU, pageable ones are staged
 * through device memory in chunks.  Particle ids are
 * assigned consecutively from the context's id counter.  The FP32 path stores
 * x as (cell, FP32 offset) and u, qw in FP32.  Errors: PIC_EINVAL (x outside
 * [-g, nr+g] x [0, nth] with g = n_filt+2, qw == 0, on the FP32 path |qw|
 * outside [2^-100, 2^100]), PIC_ECAPACITY. */
int pic_load_particles(pic_ctx *c, int64_t n, const double *x1, const double *x2,
                       const double *u_r, const double *u_th, const double *u_ph,
                       const double *qw, int32_t mem);

/* Enqueue nsteps full time steps (gather, push, move, deposit, filter, field
 * update, lossy layer, injection).  Every sort_interval steps the particles
 * are sorted (FP32: by tile, removing deleted ones; FP64: compacted), which
 * synchronises the stream once to read the live count; between sorts the
 * steps are only enqueued.  Returns errors latched by earlier steps. */
int pic_step(pic_ctx *c, int32_t nsteps);

/* Fields: out6 = 6 planes [E_r, E_th, E_ph, B_r, B_th, B_ph], each
 * (nr+1) x (nth+1) FP64, row-major [i][j]; index (i, j) of a component means its
 * staggered point of Eq. (offseteq) (e.g. E_r[i][j] is at (i+1/2, j)); entries
 * outside a component's range are 0.  which: PIC_FIELDS_PLASMA, the stored
 * plasma field; PIC_FIELDS_TOTAL, plasma plus the analytic field of the
 * descriptor's vacuum kind at time step * dt (Sec. 5.2; every grid point lies
 * at r >= r0, where the outside analytic field applies).  *n receives the
 * element count 6*(nr+1)*(nth+1); out6 == NULL only queries *n. */
int pic_get_fields(pic_ctx *c, int32_t which, double *out6, int64_t *n, int32_t mem);

/* Replace the plasma fields (layout of pic_get_fields; other entries ignored). */
int pic_set_fields(pic_ctx *c, const double *in6, int32_t mem);

/* Charge fluxes of the last step after filtering: 3 planes [F_r, F_th, F_ph] of
 * (nr+2g+1) x (nth+1) FP64 with row index i+g, g = n_filt + 2 (ghost rows
 * inside the conductors).  *n receives the element count; out3 == NULL queries. */
int pic_get_flux(pic_ctx *c, double *out3, int64_t *n, int32_t mem);

/* Charge density in integral form (Sec. 2, Eq. Jcons): Q at every node, the
 * sum over live particles of qw times the area (CIC) weight of the node in
 * grid coordinates; with filtered != 0, after the n_filt 1-2-1 passes with
 * the polar fold that the current also receives (App. B), i.e. the charge
 * Gauss's law conserves.  Layout of one pic_get_flux plane: (nr+2g+1) x
 * (nth+1) FP64, row index i+g.  *n receives the element count; out == NULL
 * queries. */
int pic_get_charge(pic_ctx *c, int32_t filtered, double *out, int64_t *n, int32_t mem);

/* Grid coordinates of physical positions (Sec. 3.2): x1 = f_r^-1(r),
 * x2 = f_th^-1(th) for n points, computed on the device; r, th, x1, x2 are n
 * FP64 values each, host or device per mem.  Use it to load particles given
 * as (r, theta). */
int pic_grid_coords(pic_ctx *c, int64_t n, const double *r, const double *th, double *x1, double *x2,
                    int32_t mem);

/* Live particles, any order, FP64 (FP32 state is widened exactly: x1 = cell +
 * offset).  *n in: capacity of the buffers; out: live count.  A NULL x1 only
 * queries the count.  id may be NULL. */
int pic_get_particles(pic_ctx *c, int64_t *n, double *x1, double *x2, double *u_r,
                      double *u_th, double *u_ph, double *qw, int64_t *id, int32_t mem);

/* Live particles written to caller-owned DEVICE buffers without any device
 * allocation (the paper has no counterpart: this serves callers that must not
 * have the library call cudaMalloc, e.g. code under its own device-memory
 * pool, or a host loop that cannot afford an allocation's synchronisation).
 * Unlike pic_get_particles it leaves the context as it is and writes the live
 * particles in slot order.  *n in: capacity of the buffers (elements); out:
 * the live count (if that exceeds the capacity, nothing beyond the capacity
 * is written and PIC_EINVAL is returned).  id may be NULL.  Scratch is a
 * static 4 MiB device array per GPU, which bounds the context to at most 2^28
 * particle slots (PIC_EINVAL beyond).  The first call on a device looks up the
 * array's address, so make it outside any stream capture; calls that overlap
 * on the GPU share the array and race.  Every output pointer must be memory
 * of the context's device (or managed memory): anything else is refused with
 * PIC_EINVAL before a kernel runs.  Synchronises the context's stream and,
 * like the other getters, returns errors latched by earlier steps. */
int pic_get_particles_noalloc(pic_ctx *c, int64_t *n, double *x1, double *x2, double *u_r,
                              double *u_th, double *u_ph, double *qw, int64_t *id);

/* Live particle count and total kinetic energy only (one streaming reduction,
 * synchronises); cheaper than pic_get_moments, which also deposits the charge. */
int pic_get_live(pic_ctx *c, int64_t *live, double *kinetic_energy);

/* Diagnostics (synchronises).  The Gauss residual is relative to the snapshot
 * taken by the first pic_step or by pic_gauss_snapshot. */
int pic_get_moments(pic_ctx *c, pic_moments *out);

/* Spin-down luminosity profile (Sec. 5.3, the luminosity of Fig. 7d):
 * L[i], i = 0..nr, the radial Poynting flux (E x B)_r (c = 1) of the total
 * field -- plasma plus the analytic field at the current time -- through the
 * sphere of node radius r_i, for 1 <= i <= nr - 1 (L[0] = L[nr] = 0).  The
 * staggered components are averaged to the centres of the meridional cells on
 * the sphere, each cell weighted by its exact area 2 pi r_i^2 (cos th_j -
 * cos th_{j+1}).  *n receives nr + 1; L == NULL only queries *n.  L is host or
 * device memory per mem.  For the force-free monopole wind of surface field B0
 * and angular velocity Omega the profile is (8 pi / 3) B0^2 r0^4 Omega^2 at
 * every radius. */
int pic_get_luminosity(pic_ctx *c, double *L, int64_t *n, int32_t mem);
int pic_gauss_snapshot(pic_ctx *c);

/* Step counter and id counter (for replaying a saved state). */
int pic_set_clock(pic_ctx *c, int64_t step, int64_t next_id);

/* Per-kernel timing of later steps with CUDA events on the context's stream:
 * enable = 1 starts accumulating; pic_get_profile writes the mean milliseconds
 * per launch of [particle kernel, deposit reduction, filter, field update,
 * injection, sort] into ms6 and the number of timed steps into *steps. */
int pic_profile(pic_ctx *c, int32_t enable);
int pic_get_profile(pic_ctx *c, double *ms6, int64_t *steps);

/* Ties of the azimuth branch at the polar axis (Sec. 3.3; the azimuthal flux
 * of a move is qw times the swept azimuth over 2 pi).  A move that carries a
 * particle across the polar axis (P_x < 0, the displaced point's coordinate
 * along the old cylindrical radius) sweeps an azimuth whose sign is that of
 * u_ph, and the two signs differ by up to 2 pi, i.e. by up to the particle's
 * whole charge in the azimuthal flux.  When |u_ph| <= 2^-13 |u| the sign is
 * set by the rounding of a nearly vanishing u_ph and either branch is a valid
 * result.  Every context counts its ties (pic_moments.axis_ties) and logs the
 * first 65536 as (step, id, sign = +1 or -1, the branch taken).
 *
 * pic_get_axis_ties: *n in: capacity of the host arrays; out: ties logged.
 * steps == NULL only queries *n.  signs may be NULL.
 * pic_set_axis_hints: n host entries (step, id, sign) that fix the branch of
 * those ties when this context meets them (a replay of another run follows
 * that run's branches); any previous table is replaced, n = 0 removes it.
 * Ties the table does not list keep their own branch. */
int pic_get_axis_ties(pic_ctx *c, int64_t *n, int64_t *steps, int64_t *ids, int32_t *signs);
int pic_set_axis_hints(pic_ctx *c, int64_t n, const int64_t *steps, const int64_t *ids, const int32_t *signs);

/* Failure detection without a fault: the device-side waits of the library
 * (the tile kernel's wait for its field window, Sec. 3 of the design's
 * hot path) poll a bounded number of times and then latch PIC_ETIMEOUT
 * instead of hanging.  This runs that wait on its own in one small kernel on
 * `stream`: with arrive_first = 0 nothing completes the awaited phase, the
 * wait gives up after `polls` polls and the call returns PIC_ETIMEOUT; with
 * arrive_first = 1 the phase completes first and the call returns PIC_OK.
 * Either way the kernel ends and no context is affected.  The paper has no
 * counterpart; it serves callers and tests that check the failure path. */
int pic_wait_selftest(int64_t polls, int32_t arrive_first, void *stream);

/* Number of kernels this context has launched so far (every launch of the
 * library's own kernels, all phases); *n receives the count. */
int pic_get_launches(pic_ctx *c, int64_t *n);

/* Advance n independent contexts by nsteps each, batched (an ensemble of
 * independent simulations with uneven grids and particle counts).
 *
 * All FP32 members: each phase of a step is ONE kernel launch over the blocks
 * of every member that takes part in it -- the tile kernel once per tile
 * shape and specialisation present, then the flux conversion, each filter
 * pass, the three Yee sub-steps, the lossy layer, the axis ghosts and FP32
 * copies, and the injection phases -- with the members' arguments for each
 * step in a device table; the steps up to the next sort of any member are
 * captured into one CUDA graph, launched once.  Each member's tile sort runs
 * between graphs when its own sort interval comes due, so every member takes
 * the same steps and sorts as in its own pic_step run, with bit-identical
 * results.
 *
 * Any FP64 member: every member's steps are captured into the graph on a
 * parallel branch of their own (one kernel launch per phase per member).
 *
 * ctxs: n distinct contexts on one device (host array of handles, read during
 * the call only).  kernels: may be NULL; receives the number of kernel
 * launches the call enqueued (graph kernel nodes and sorts).  Each member's
 * own launch count (pic_get_launches) advances by the launches its own
 * pic_step run would take: a batched launch counts once for every member it
 * serves.  Each member's own stream waits for the graph.  Errors: PIC_EINVAL
 * (NULL or repeated members, several devices, nsteps < 0), PIC_ENOMEM,
 * PIC_ECUDA; errors latched in any member are returned. */
int pic_ensemble_step(pic_ctx *const *ctxs, int32_t n, int32_t nsteps, int64_t *kernels);

/* Pick the FP32 path's tile shape and sort interval by measurement: every
 * candidate (3 tile shapes x sort intervals 5, 10, 20, 40) runs trial_steps
 * steps on a clone of the context (the context itself does not advance), and
 * the fastest mean step time wins and is applied to the context.  The chosen
 * values are returned in *sort_interval and *tile_shape (either may be NULL).
 * Costs about 12 clones' worth of device memory and time: meant for the
 * small members of an ensemble.  FP64 contexts: PIC_EINVAL. */
int pic_autotune(pic_ctx *c, int32_t trial_steps, int32_t *sort_interval, int32_t *tile_shape);

/* The same choice for an ensemble as a whole: every candidate (3 tile shapes x
 * sort intervals 10, 20, 40) runs on clones of all n members through
 * pic_ensemble_step (one sort cycle of warm-up, then max(trial_steps, 2 x
 * interval) steps timed on the host clock, which includes the batched step's
 * host work), and the fastest pair is applied to every member: one shape and
 * one interval keep each step's tile launches and sorts to one batch each.
 * The members do not advance.  Holds a clone of every member at once (about
 * twice the ensemble's device memory).  ctxs: n distinct FP32 contexts on one
 * device.  Errors: PIC_EINVAL (NULL, repeated or FP64 members, trial_steps <
 * 1), PIC_ENOMEM, PIC_ECUDA. */
int pic_autotune_ensemble(pic_ctx *const *ctxs, int32_t n, int32_t trial_steps, int32_t *sort_interval,
                          int32_t *tile_shape);

/* Release every device buffer of the context.  NULL is allowed. */
int pic_destroy(pic_ctx *c);

/* ---- one simulation split into radial slabs ---------------------------------
 * The grid decomposition the paper parallelises over MPI (Sec. 2, Overview;
 * the scaling discussion of Sec. 6): the nr rows are cut into nslabs
 * contiguous radial slabs, each held by a context of its own on the current
 * device.  Every step exchanges between neighbouring slabs: the field rows
 * next to each interface after each Yee sub-step (the gather and the curl read
 * one row across it), the charge flux the particles deposit into the
 * neighbour's rows (summed back into the owner before the N_filt filter
 * passes, which then read N_filt + 2 ghost rows), and the particles that
 * crossed the interface (at most one cell per step, by the Courant limit).
 * Each exchange is a contiguous block copied on the stream, the message a
 * point-to-point send would carry between GPUs.  The results are those of one
 * context over the whole grid (pic_init_grid): on the FP64 path up to the
 * order of the FP64 current sums; on the FP32 path bit for bit (every slab
 * deposits in one shared fixed-point quantum and the neighbours' int64 sums
 * are added exactly before the conversion to FP64). */
typedef struct pic_slabs pic_slabs;

/* d: the whole grid's descriptor (as for pic_init_grid; dt <= 0 takes the
 * whole grid's Courant step).  rows: nslabs + 1 slab boundaries in global
 * rows, 0 = rows[0] < ... < rows[nslabs] = nr, or NULL for equal slabs.  Every
 * slab needs at least 2 (n_filt + 2) + 2 rows, and the lossy layer must lie in
 * the last slab.  Errors: PIC_EINVAL (bad descriptor or rows), PIC_ENOMEM,
 * PIC_ECUDA. */
int pic_slabs_init(pic_slabs **out, const pic_desc *d, int32_t nslabs, const int32_t *rows, void *stream);

/* Append n particles in global grid coordinates (as pic_load_particles; ids
 * are consecutive over the whole load); each goes to the slab of its row. */
int pic_slabs_load_particles(pic_slabs *g, int64_t n, const double *x1, const double *x2, const double *u_r,
                             const double *u_th, const double *u_ph, const double *qw, int32_t mem);

/* nsteps full time steps of the whole grid (synchronises once per step to
 * hand over the migrating particles).  Returns errors latched in any slab. */
int pic_slabs_step(pic_slabs *g, int32_t nsteps);

/* The whole grid's fields, fluxes, particles (global x1) and moments, in the
 * layouts of pic_get_fields, pic_get_flux, pic_get_particles and
 * pic_get_moments, assembled from the rows each slab owns. */
int pic_slabs_get_fields(pic_slabs *g, int32_t which, double *out6, int64_t *n, int32_t mem);
int pic_slabs_get_flux(pic_slabs *g, double *out3, int64_t *n, int32_t mem);
int pic_slabs_get_particles(pic_slabs *g, int64_t *n, double *x1, double *x2, double *u_r, double *u_th,
                            double *u_ph, double *qw, int64_t *id, int32_t mem);
int pic_slabs_get_moments(pic_slabs *g, pic_moments *out);

/* Release every slab.  NULL is allowed. */
int pic_slabs_destroy(pic_slabs *g);

/* Message of the last failed call on this thread ("" if none). */
const char *pic_last_error(void);

/* sizeof(pic_desc) and sizeof(pic_moments) as compiled into the library, for
 * bindings that mirror the two structs (no device work). */
void pic_struct_sizes(int64_t *desc_bytes, int64_t *moments_bytes);

#ifdef __cplusplus
}
#endif
#endif

// pic_internal.h -- host-side context of the library and the launchers each
// translation unit provides.  Not part of the public C-ABI (include/picsar.h).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "picsar.h"  // include/ is on the include path
#include "pic_common.cuh"

namespace pic {

// FP64 particle arrays (structure of arrays, 56 B per particle with the id)
struct Parts64 {
  double *x1 = nullptr, *x2 = nullptr, *ur = nullptr, *ut = nullptr, *up = nullptr, *qw = nullptr;
  int64_t *id = nullptr;
};
// FP32 particle arrays: packed cell (i + CELL_BIAS) << 16 | j, FP32 offsets in
// the cell, FP32 momentum and charge; 28 B per particle plus the 8 B id
struct Parts32 {
  uint32_t *cell = nullptr;
  float *dx = nullptr, *dy = nullptr, *ur = nullptr, *ut = nullptr, *up = nullptr, *qw = nullptr;
  int64_t *id = nullptr;
};
constexpr int CELL_BIAS = 1024;

// device counters (one int64 array)
enum Counter { CNT_DELETED = 0, CNT_INJECTED = 1, CNT_LIVE = 2, CNT_SMAX = 3, CNT_GMAX = 4,
               CNT_QMAX = 5, CNT_SORTED = 6, CNT_QEXP = 7, CNT_CAPPED = 8, CNT_TIES = 9, CNT_N };
constexpr int64_t TIE_LOG = 1 << 16;  // axis-crossing ties logged per context

// FP32 path fixed-point deposit.  One flux unit is 2^(e - KFIX) with e =
// ceil(log2 max |qw|) over every charge the context has held (loaded or
// injected), kept on the device in d_cnt[CNT_QEXP]: the loading and
// injection kernels raise it with atomicMax, the deposit and the conversion
// to FP64 read it, so no flux term exceeds 2^KFIX units and the quantum
// follows the charges without any host round trip.  e is clamped to
// [QEXP_MIN, QEXP_MAX]; QEXP_NONE marks a context that has held no charge.
constexpr int KFIX = 36;
constexpr int QEXP_MIN = -90, QEXP_MAX = 100;
constexpr long long QEXP_NONE = -1000000;

// ceil(log2 a) of a charge magnitude a > 0, clamped to [QEXP_MIN, QEXP_MAX]
__device__ inline int charge_exp(float a) {
  int e;
  const float m = frexpf(a, &e);  // a = m 2^e, 0.5 <= m < 1
  if (m == 0.5f) --e;             // a power of two: log2 a = e - 1 exactly
  return e < QEXP_MIN ? QEXP_MIN : (e > QEXP_MAX ? QEXP_MAX : e);
}

// Raise the context's exponent to the warp's largest e (QEXP_NONE: no
// charge).  Every lane of the warp must call it.  The plain read first
// skips the atomic in the common case of a bound already reached.
__device__ inline void raise_qexp(long long *qexp, int e) {
  e = __reduce_max_sync(0xffffffffu, e);
  if ((threadIdx.x & 31) == 0 && e > *(volatile long long *)qexp) atomicMax(qexp, (long long)e);
}

// the exponent as the kernels use it (a context with no charge yet: 0)
__device__ inline int qexp_value(const long long *qexp) {
  const long long e = *qexp;
  return e < QEXP_MIN ? 0 : (int)e;
}
// device double accumulators
enum Accum { ACC_KIN = 0, ACC_FIELD = 1, ACC_CHARGE = 2, ACC_N };

// FP32 path: particles are counting-sorted by cell, cells numbered tile by
// tile (tile-major, row-major inside a tile), so each tile's particles form
// one contiguous range ordered by cell
struct Tiles {
  int TI = 16, TJ = 16;          // tile size in cells
  int nti = 0, ntj = 0, ntiles = 0;
  int row0 = 0;                   // first tile row (cell index)
  int tc = 256;                   // cells per tile, TI * TJ
  int64_t nbins = 0;              // ntiles * tc cell bins + 1 bin of removed particles
  int64_t *start = nullptr;       // nbins + 1 bin starts: tile t is [start[t tc], start[(t+1) tc])
  int64_t *cursor = nullptr;      // nbins + 1 counts, then scatter cursors
  int64_t *bsum = nullptr;        // 2 (nbins / SCAN_CHUNK + 2) partial sums of the scan
  int64_t sorted_end = 0;         // particles [0, sorted_end) are binned
  // work units of the tile kernel: each sort splits a tile's bin into units
  // of at most `unit` particles, one CTA each (the deposit sums are exact, so
  // the split changes no result)
  int64_t unit = 0;               // particles per work unit
  int64_t nunits = 0;             // work units of the binned particles
  long long *units = nullptr;     // per unit: tile << 32 | index of the unit within its tile
  int64_t units_cap = 0;
  int64_t *ucount = nullptr;      // per tile: its units, then their exclusive scan (ntiles + 1)
  int64_t *usum = nullptr;        // partial sums of that scan
};
constexpr int SCAN_CHUNK = 4096;  // bins per block of the multi-block scan

// ---- batched launches over the members of an ensemble ------------------------
// One launch covers the blocks of several members: block b of the grid serves
// entry blk[b].x of the step's argument table as that member's block blk[b].y
// (one load per block; the map lives in device memory).
struct EnsList {
  const int2 *blk = nullptr;
};

enum ProfSlot { PROF_PARTICLES = 0, PROF_REDUCE = 1, PROF_FILTER = 2, PROF_FIELDS = 3, PROF_INJECT = 4,
                PROF_SORT = 5, PROF_N };

// One FP32 member at one step as the batched grid kernels read it: the
// member's grid and arrays, the flux buffers as the step starts, after its
// filter passes and their scratch, and the step's injection.
struct EnsFieldArg {
  Grid G;
  double *f[6];
  double *Fin[3], *Ftmp[3], *Fout[3];  // flux written by the deposit; filter scratch; flux the E update reads
  float *f32[6];
  long long *acc[3];
  size_t grid_elems;
  long long *cnt;
  long long *qexp;                     // the fixed-point exponent counter
  double *sig;                         // two buffers of nth + 1
  Parts32 p32;
  int64_t inj_base, inj_id0;           // first slot and id of the step's injected pairs
  double t_inj;                        // time at which the injection reads the field
  double f_inj, inject_q;
  uint64_t inject_seed, inj_step;
  int inject, npp, inject_smooth, n_filt;
  int lossy_i0;                        // first row of the lossy layer (-1: none)
};

// kinds of batched grid launch (block counts per member: ens_blocks)
enum EnsKind { ENS_FLUX = 0, ENS_FILTER, ENS_NODES, ENS_LOSSY, ENS_GHOSTS, ENS_COPY32, ENS_SIGMA, ENS_WRITE,
               ENS_NKIND };

}  // namespace pic

struct pic_ctx {
  pic_desc d{};
  cudaStream_t stream = nullptr;
  int device = 0;
  pic::Grid G{};
  double *metric_buf = nullptr;
  size_t grid_elems = 0;  // elements of one padded grid array
  double *f[6] = {};      // plasma fields (FP64)
  double *F[3] = {};      // fluxes of the current step (FP64, after filtering)
  double *Ft[3] = {};     // filter double buffer
  float *f32[6] = {};     // FP32 gather copies (FP32 path)
  float *r_n32 = nullptr; // f_r(i) per padded row, FP32 (FP32 path)
  float2 *th_n32 = nullptr; // (sin, cos) of the linear map's node angle per padded column (FP32 path)
  long long *acc[3] = {}; // fixed-point flux accumulators (FP32 path)
  alignas(64) unsigned char tile_maps[3][6 * 128] = {}; // FP32: field tensor maps per tile shape (TMA)
  unsigned char *d_tile_maps = nullptr;  // the same maps in device memory (batched ensemble launches)
  double *Q = nullptr, *Qa = nullptr, *Qt = nullptr, *gsnap = nullptr;
  bool have_snap = false;
  double *sig = nullptr;  // injection: surface charge per cell, two buffers of nth + 1 (smoothing)
  // particles
  int64_t cap = 0, n_used = 0;
  pic::Parts64 p64, q64;  // current and alternate (compaction) buffers
  pic::Parts32 p32, q32;
  pic::Tiles tiles;
  void *scratch = nullptr;  // compaction / sort scratch
  size_t scratch_bytes = 0;
  int *d_err = nullptr;
  long long *d_cnt = nullptr;
  // the fixed-point exponent counter: d_cnt + CNT_QEXP, or the one the
  // radial slabs of a grid share (every slab's fluxes in one quantum)
  long long *qexp = nullptr;
  double *d_acc = nullptr;
  long long *h_pinned = nullptr;  // pinned host mirror for small reads
  // axis-crossing ties: the log of this context and the hints it follows
  int64_t *tie_step = nullptr, *tie_id = nullptr;
  int8_t *tie_sign = nullptr;
  int64_t *hint_step = nullptr, *hint_id = nullptr;
  int8_t *hint_sign = nullptr;
  int64_t nhint = 0;
  int64_t step = 0, next_id = 0;
  int64_t launches = 0;  // kernels launched by this context
  int host_err = 0;
  int steps_since_sort = 0;
  bool need_sort = false;
  bool small_steps = false; // FP32: the grid bounds the move's series arguments (series without fallback)
  bool mix_sort = true;    // FP32: the next sort orders by cell and mixes each tile's bin
  // profiling: one start/stop event pair per phase per step, read back lazily
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;           // recorded events, pairs per phase
  std::vector<int> ev_slot;                   // phase of each pair
  size_t ev_used = 0;
  double prof_ms[pic::PROF_N] = {};
  int64_t prof_launch[pic::PROF_N] = {};
  int64_t prof_steps = 0;
};

namespace pic {
// fields.cu
void fields_b_half(pic_ctx *c);
void fields_e_full(pic_ctx *c);
void fields_finish(pic_ctx *c);        // lossy layer + axis ghosts (+ FP32 copies)
void fields_filter(pic_ctx *c);        // n_filt passes on F
void fields_fill_ghosts(pic_ctx *c);   // axis ghosts (+ FP32 copies) (after pic_set_fields)
void fields_copy32(pic_ctx *c);        // FP32 gather copies of the fields (FP32 path)
void inject(pic_ctx *c, double t);     // surface pairs into slots [n_used, n_used + 2 npp nth)
void moments(pic_ctx *c, bool snapshot, pic_moments *out);
void luminosity(pic_ctx *c, double t, double *L);  // nr + 1 device values (Sec. 5.3)
void filter_array(pic_ctx *c, double *a, double *tmp, int half_j, int sign, int passes);
// Gauss law (G - Qbar against the snapshot, into d_cnt[CNT_GMAX/QMAX]) over
// local rows ilo..imax, with Q, Qa already deposited and filtered
void gauss_rows(pic_ctx *c, int ilo, int imax, bool snapshot);
void field_energy_rows(pic_ctx *c, int imax);  // adds rows 0..imax to d_acc[ACC_FIELD]
// particles64.cu
void particles64(pic_ctx *c, double t);
int64_t compact64(pic_ctx *c);         // stable removal of dead slots; returns live count
void charge64(pic_ctx *c, double *Q, double *Qa);
void reduce_particles64(pic_ctx *c);   // kinetic energy, live count, total charge
// batched launches over ensemble members (fields.cu); blocks: the launch's grid
int ens_blocks(const pic_ctx *c, int kind);  // blocks one member needs in a launch of that kind
void ens_fill_field_arg(const pic_ctx *c, EnsFieldArg *a);  // the member's arrays (not the step's values)
void ens_filter(const EnsFieldArg *tab, const EnsList &L, int blocks, int pass, cudaStream_t s);
void ens_b_half(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s);
void ens_e_full(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s);
void ens_lossy(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s);
void ens_ghosts(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s);
void ens_copy32(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s);
void ens_inject_sigma(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s);
void ens_inject_smooth(const EnsFieldArg *tab, const EnsList &L, int blocks, int pass, cudaStream_t s);
void ens_inject_write(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s);
// particles32.cu
int tiles32_setup(pic_ctx *c);         // tensor maps of the field window (FP32 path, at creation)
// batched tile kernel: members grouped by kind (specialisation x tile shape)
constexpr int ENS_TILE_KINDS = 9;
size_t ens_tile_arg_bytes();
int ens_tile_kind(const pic_ctx *c);
int64_t ens_tile_blocks(const pic_ctx *c);           // 0 when the member holds no particles
void ens_tile_arg(pic_ctx *c, double t, void *out);  // the member's tile-kernel arguments at time t
// launches the tile kernel of one kind over n members (host array of their
// arguments, ens_tile_arg_bytes() each, and their block counts); returns the
// number of kernels launched (members are taken in groups of up to 48)
int ens_tiles32(int kind, const void *args, const int64_t *blocks, int n, cudaStream_t s);
void ens_flux_from_acc(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s);
// the tile sort of m FP32 contexts at once on stream st (each launch serves
// every member; one read-back, one synchronisation); the staging buffers
// persist in sc between calls.  *kernels: the kernels launched.
struct EnsSortScratch {
  unsigned char *h = nullptr, *d = nullptr;
  size_t cap = 0;
};
int ens_sort32(pic_ctx *const *cs, int m, cudaStream_t st, EnsSortScratch &sc, int64_t *kernels);
void ens_sort_scratch_free(EnsSortScratch &sc);
void particles32(pic_ctx *c, double t);
void flux_from_acc(pic_ctx *c);        // fixed point -> FP64 fluxes, clears the accumulators
int64_t sort32(pic_ctx *c);            // tile sort + removal; returns live count
void charge32(pic_ctx *c, double *Q, double *Qa);
void reduce_particles32(pic_ctx *c);
// the tie log and hints of a context for the step it is taking
inline AxisTies axis_ties(const pic_ctx *c);
}  // namespace pic

inline pic::AxisTies pic::axis_ties(const pic_ctx *c) {
  AxisTies X;
  X.hstep = c->hint_step; X.hid = c->hint_id; X.hsign = c->hint_sign; X.nh = c->nhint;
  X.lstep = c->tie_step; X.lid = c->tie_id; X.lsign = c->tie_sign; X.lcap = TIE_LOG;
  X.count = c->d_cnt + CNT_TIES;
  X.step = c->step;
  return X;
}

// error plumbing (api.cu)
int pic_fail(int code, const std::string &msg);
int pic_cuda_check(cudaError_t e, const char *what);
int pic_latch_status(pic_ctx *c);  // read the device error word, return the context's status
int pic_desc_defaults(pic_desc *d);  // fill the zero defaults and check the descriptor
// a context over rows [i0, i0 + d.nr) of a grid of nr_glob rows (api.cu)
int pic_create_context(pic_ctx **out, const pic_desc &d, void *stream, int i0, int nr_glob, int open_lo, int open_hi);
int pic_grow_particles(pic_ctx *c, int64_t new_cap);  // keep [0, n_used), reallocate
int pic_compact(pic_ctx *c);                          // remove free slots (sort on the FP32 path)
// stepping internals of api.cu that the ensemble (ensemble.cu) drives
void pic_step_body(pic_ctx *c);                        // enqueue one full step on c->stream
int pic_prepare_steps(pic_ctx *c, int steps);          // host work before `steps` steps can be enqueued blindly
int pic_set_tiles(pic_ctx *c, int shape);              // re-bin an FP32 context for another tile shape
int pic_clone_context(pic_ctx *c, pic_ctx **out);      // a new context holding the same fields, particles and clock
int pic_reserve(pic_ctx *c, int64_t need);            // capacity for at least `need` particle slots
#define PIC_CUDA(call)                                          \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return pic_cuda_check(e_, #call);    \
  } while (0)

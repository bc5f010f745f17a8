// slabs.cu -- one simulation split into radial slabs (the grid decomposition
// the paper runs over MPI, Sec. 2), each slab a context of its own, with the
// exchanges a step needs between neighbouring slabs:
//
//   * field halo: after each Yee sub-step, the rows next to an interface are
//     copied to the neighbour's ghost rows (the gather reads one ghost row on
//     each side, the curl one row of E or B across the interface);
//   * flux halo: the charge a slab's particles deposit into rows owned by the
//     neighbour is summed back into the owner, then the owner's rows are copied
//     out again to N_filt + 2 ghost rows, which the filter (App. B) reads;
//   * particle migration: a particle moves at most one cell per step
//     (Courant), so after the push each slab hands the particles that left its
//     rows to the neighbour on that side.
//
// Every message is one contiguous block (whole padded rows, or a packed list
// of particles), staged in a buffer of the receiver: on one GPU a device
// copy carries it, on several GPUs (one slab per rank) the same blocks would
// be point-to-point sends.  Particles keep global grid coordinates; a slab's
// kernels subtract its first row only to index its arrays, so each particle
// step is the same arithmetic as on the whole grid.
//
// Both particle paths.  The FP64 path sums the neighbours' FP64 flux rows
// (results equal the whole grid's up to the order of the FP64 atomic sums).
// The FP32 path keeps whole-grid rows in each particle's packed cell (a
// slab's kernels see its arrays through a shifted row offset), shares one
// fixed-point quantum among all slabs and sums the neighbours' int64
// fixed-point rows before the conversion, so its fluxes are the whole
// grid's exactly.
#include <algorithm>
#include <cstring>
#include <vector>

#include "pic_internal.h"

using namespace pic;

struct pic_slabs {
  pic_desc d{};                 // the whole grid (defaults filled)
  int S = 0;
  std::vector<int> a;           // slab s holds global rows [a[s], a[s+1])
  std::vector<pic_ctx *> ctx;
  cudaStream_t stream = nullptr;
  double *stage = nullptr;      // one halo message (g + 1 padded rows)
  size_t stage_elems = 0;
  Parts64 box[2];               // particle messages: [0] to the lower, [1] to the upper neighbour
  int64_t box_cap = 0;
  Parts32 box32[2];             // the same for the FP32 path (cells in whole-grid rows)
  int64_t box32_cap = 0;
  long long *d_box = nullptr;   // their counts
  long long *h_box = nullptr;   // pinned mirror
  int64_t step = 0, next_id = 0;
  bool have_snap = false;
};

namespace {

template <class T>
__global__ void k_add(T *__restrict__ dst, const T *__restrict__ src, size_t n) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
    dst[k] += src[k];
}

// start of padded row i (local) of a grid array (FP64 or int64 fixed point)
template <class T>
inline T *row_ptr(const pic_ctx *c, T *a, int i) { return a + (size_t)(i + c->G.PI) * c->G.LD; }

template <class T>
int copy_rows(pic_slabs *g, T *dst, const T *src, int rows, const pic_ctx *c) {
  PIC_CUDA(cudaMemcpyAsync(dst, src, (size_t)rows * c->G.LD * sizeof(T), cudaMemcpyDeviceToDevice, g->stream));
  return PIC_OK;
}

// ghost rows of one array across the interface lo | hi: H rows each way
int halo_set(pic_slabs *g, pic_ctx *lo, pic_ctx *hi, double *alo, double *ahi, int H) {
  const int n = lo->G.nr;
  int e;
  if ((e = copy_rows(g, row_ptr(hi, ahi, -H), row_ptr(lo, alo, n - H), H, lo))) return e;
  return copy_rows(g, row_ptr(lo, alo, n), row_ptr(hi, ahi, 0), H, lo);
}

// deposits in ghost rows summed back into the owner's rows (through the
// staging buffer, as a received message would be), then the owner's rows
// copied out to the ghosts again (FP64 fluxes and charges, or the FP32
// path's int64 fixed-point sums, which add exactly)
template <class T>
int halo_sum(pic_slabs *g, pic_ctx *lo, pic_ctx *hi, T *alo, T *ahi) {
  static_assert(sizeof(T) == sizeof(double), "the staging buffer holds 8-byte elements");
  const int n = lo->G.nr, gg = lo->G.g;
  const size_t LD = lo->G.LD;
  const unsigned blocks = 4 * 152;
  T *stage = reinterpret_cast<T *>(g->stage);
  int e;
  // hi's rows -g..-1 belong to lo (its rows n-g..n-1)
  if ((e = copy_rows(g, stage, row_ptr(hi, ahi, -gg), gg, lo))) return e;
  ++lo->launches, k_add<T><<<blocks, 256, 0, g->stream>>>(row_ptr(lo, alo, n - gg), stage, (size_t)gg * LD);
  // lo's rows n..n+g belong to hi (its rows 0..g)
  if ((e = copy_rows(g, stage, row_ptr(lo, alo, n), gg + 1, lo))) return e;
  ++hi->launches, k_add<T><<<blocks, 256, 0, g->stream>>>(row_ptr(hi, ahi, 0), stage, (size_t)(gg + 1) * LD);
  if ((e = copy_rows(g, row_ptr(hi, ahi, -gg), row_ptr(lo, alo, n - gg), gg, lo))) return e;
  return copy_rows(g, row_ptr(lo, alo, n), row_ptr(hi, ahi, 0), gg + 1, lo);
}

// field ghosts of the listed components at every interface
int exchange_fields(pic_slabs *g, const int *comps, int nc) {
  for (int s = 0; s + 1 < g->S; ++s)
    for (int k = 0; k < nc; ++k) {
      const int e = halo_set(g, g->ctx[s], g->ctx[s + 1], g->ctx[s]->f[comps[k]], g->ctx[s + 1]->f[comps[k]], 2);
      if (e) return e;
    }
  return PIC_OK;
}

// particles whose cell left the slab through an open side go to that side's
// message; their slot is freed
// (a particle that finds its message full stays, still counted: the host
// enlarges the message and runs the pass again)
__global__ void k_emigrate(Grid G, Parts64 P, int64_t n, Parts64 lo, Parts64 hi, int64_t cap, long long *cnt) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double q = P.qw[k];
  if (q == 0.0) return;
  const int ci = (int)floor(P.x1[k]) - G.i0;
  int side = -1;
  if (G.open_lo && ci < 0) side = 0;
  if (G.open_hi && ci >= G.nr) side = 1;
  if (side < 0) return;
  const long long d = atomicAdd(reinterpret_cast<unsigned long long *>(cnt + side), 1ull);
  if (d >= cap) return;
  Parts64 &B = side ? hi : lo;
  B.x1[d] = P.x1[k]; B.x2[d] = P.x2[k];
  B.ur[d] = P.ur[k]; B.ut[d] = P.ut[k]; B.up[d] = P.up[k];
  B.qw[d] = q; B.id[d] = P.id[k];
  P.qw[k] = 0.0;
}

__global__ void k_immigrate(Parts64 P, int64_t base, Parts64 B, int64_t m) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= m) return;
  const int64_t d = base + k;
  P.x1[d] = B.x1[k]; P.x2[d] = B.x2[k];
  P.ur[d] = B.ur[k]; P.ut[d] = B.ut[k]; P.up[d] = B.up[k];
  P.qw[d] = B.qw[k]; P.id[d] = B.id[k];
}

// FP32 path: the same hand-over (packed cells hold whole-grid rows)
__global__ void k_emigrate32(Grid G, Parts32 P, int64_t n, Parts32 lo, Parts32 hi, int64_t cap, long long *cnt) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float q = P.qw[k];
  if (q == 0.f) return;
  const uint32_t c = P.cell[k];
  const int ci = (int)(c >> 16) - CELL_BIAS - G.i0;  // the slab's own row
  int side = -1;
  if (G.open_lo && ci < 0) side = 0;
  if (G.open_hi && ci >= G.nr) side = 1;
  if (side < 0) return;
  const long long d = atomicAdd(reinterpret_cast<unsigned long long *>(cnt + side), 1ull);
  if (d >= cap) return;
  Parts32 &B = side ? hi : lo;
  B.cell[d] = c;
  B.dx[d] = P.dx[k]; B.dy[d] = P.dy[k];
  B.ur[d] = P.ur[k]; B.ut[d] = P.ut[k]; B.up[d] = P.up[k];
  B.qw[d] = q; B.id[d] = P.id[k];
  P.qw[k] = 0.f;
}

__global__ void k_immigrate32(Parts32 P, int64_t base, Parts32 B, int64_t m) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= m) return;
  const int64_t d = base + k;
  P.cell[d] = B.cell[k];
  P.dx[d] = B.dx[k]; P.dy[d] = B.dy[k];
  P.ur[d] = B.ur[k]; P.ut[d] = B.ut[k]; P.up[d] = B.up[k];
  P.qw[d] = B.qw[k]; P.id[d] = B.id[k];
}

// the slab's share of an FP32 load: the cell and FP32 offsets as
// pic_load_particles forms them on the whole grid (the carry of an offset
// that rounds to 1 decides the row, and so the slab);
// counted (D.cell == NULL) or appended at base + an atomic slot; the charges
// raise the shared fixed-point exponent
__global__ void k_load_slab32(Grid G, Parts32 D, int64_t base, int64_t n, const double *x1, const double *x2,
                              const double *ur, const double *ut, const double *up, const double *qw, int64_t id0,
                              long long *cnt, int *err, long long *qexp) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int qe = (int)QEXP_NONE;
  if (k < n) {
    const double a = x1[k], b = x2[k], q = qw[k], vr = ur[k], vt = ut[k], vp = up[k];
    const bool ok = (a >= -(double)(G.n_filt + 1)) & (a < (double)(G.nr_glob + G.n_filt + 1)) & (b >= 0.0) &
                    (b <= G.nth) & (fabs(q) >= 0x1p-100) & (fabs(q) <= 0x1p100) & isfinite(vr) & isfinite(vt) &
                    isfinite(vp);
    if (!ok) {
      if (G.i0 == 0) atomicOr(err, ERR_RANGE);
    } else {
      int ci = (int)floor(a), cj = (int)floor(b);
      if (cj > G.nth - 1) cj = G.nth - 1;
      float ox = (float)(a - ci), oy = (float)(b - cj);
      if (ox >= 1.0f) { ox = 0.0f; ++ci; }
      if (oy >= 1.0f && cj < G.nth - 1) { oy = 0.0f; ++cj; }
      const int cl = ci - G.i0;
      if (!((cl < 0 && G.open_lo) || (cl >= G.nr && G.open_hi))) {  // else another slab's
        const long long s = atomicAdd(reinterpret_cast<unsigned long long *>(cnt), 1ull);
        if (D.cell) {
          const int64_t d = base + s;
          D.cell[d] = ((uint32_t)(ci + CELL_BIAS) << 16) | (uint32_t)cj;
          D.dx[d] = ox; D.dy[d] = oy;
          D.ur[d] = (float)vr; D.ut[d] = (float)vt; D.up[d] = (float)vp; D.qw[d] = (float)q;
          D.id[d] = id0 + k;
          qe = charge_exp(fabsf((float)q));
        }
      }
    }
  }
  raise_qexp(qexp, qe);  // every lane of the warp reaches this
}

// the slab's share of a particle load: rows [lo, hi) of the whole grid (the
// first slab also takes x1 < 0, the last x1 >= nr), counted (D.x1 == NULL) or
// appended at base + an atomic slot; checks as pic_load_particles
__global__ void k_load_slab(Grid G, Parts64 D, int64_t base, int64_t n, const double *x1, const double *x2,
                            const double *ur, const double *ut, const double *up, const double *qw, int64_t id0,
                            long long *cnt, int *err) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double a = x1[k], b = x2[k], q = qw[k], vr = ur[k], vt = ut[k], vp = up[k];
  const bool ok = (a >= -(double)(G.n_filt + 1)) & (a < (double)(G.nr_glob + G.n_filt + 1)) & (b >= 0.0) &
                  (b <= G.nth) & (q != 0.0) & isfinite(q) & isfinite(vr) & isfinite(vt) & isfinite(vp);
  if (!ok) { if (G.i0 == 0) atomicOr(err, ERR_RANGE); return; }
  const int ci = (int)floor(a) - G.i0;
  if ((ci < 0 && G.open_lo) || (ci >= G.nr && G.open_hi)) return;  // another slab's
  const long long s = atomicAdd(reinterpret_cast<unsigned long long *>(cnt), 1ull);
  if (!D.x1) return;
  const int64_t d = base + s;
  D.x1[d] = a; D.x2[d] = b; D.ur[d] = vr; D.ut[d] = vt; D.up[d] = vp; D.qw[d] = q; D.id[d] = id0 + k;
}

int free_box(pic_slabs *g) {
  for (Parts64 &b : g->box) {
    cudaFree(b.x1); cudaFree(b.x2); cudaFree(b.ur); cudaFree(b.ut); cudaFree(b.up); cudaFree(b.qw); cudaFree(b.id);
    b = Parts64{};
  }
  g->box_cap = 0;
  for (Parts32 &b : g->box32) {
    cudaFree(b.cell); cudaFree(b.dx); cudaFree(b.dy); cudaFree(b.ur); cudaFree(b.ut); cudaFree(b.up);
    cudaFree(b.qw); cudaFree(b.id);
    b = Parts32{};
  }
  g->box32_cap = 0;
  return PIC_OK;
}

int reserve_box32(pic_slabs *g, int64_t need) {
  if (need <= g->box32_cap) return PIC_OK;
  for (Parts32 &b : g->box32) {
    cudaFree(b.cell); cudaFree(b.dx); cudaFree(b.dy); cudaFree(b.ur); cudaFree(b.ut); cudaFree(b.up);
    cudaFree(b.qw); cudaFree(b.id);
    b = Parts32{};
  }
  g->box32_cap = 0;
  const int64_t cap = need * 2 + 4096;
  for (Parts32 &b : g->box32) {
    PIC_CUDA(cudaMalloc((void **)&b.cell, cap * sizeof(uint32_t)));
    float **f[6] = {&b.dx, &b.dy, &b.ur, &b.ut, &b.up, &b.qw};
    for (float **p : f) PIC_CUDA(cudaMalloc((void **)p, cap * sizeof(float)));
    PIC_CUDA(cudaMalloc((void **)&b.id, cap * sizeof(int64_t)));
  }
  g->box32_cap = cap;
  return PIC_OK;
}

int reserve_box(pic_slabs *g, int64_t need) {
  if (need <= g->box_cap) return PIC_OK;
  for (Parts64 &b : g->box) {
    cudaFree(b.x1); cudaFree(b.x2); cudaFree(b.ur); cudaFree(b.ut); cudaFree(b.up); cudaFree(b.qw); cudaFree(b.id);
    b = Parts64{};
  }
  g->box_cap = 0;
  const int64_t cap = need * 2 + 4096;
  for (Parts64 &b : g->box) {
    double **f[6] = {&b.x1, &b.x2, &b.ur, &b.ut, &b.up, &b.qw};
    for (double **p : f) PIC_CUDA(cudaMalloc((void **)p, cap * sizeof(double)));
    PIC_CUDA(cudaMalloc((void **)&b.id, cap * sizeof(int64_t)));
  }
  g->box_cap = cap;
  return PIC_OK;
}

// room for `extra` more slots after n_used: remove free slots first, grow if
// that is not enough
int room(pic_ctx *c, int64_t extra) {
  if (c->n_used + extra <= c->cap) return PIC_OK;
  int e = pic_compact(c);
  if (e) return e;
  return pic_reserve(c, c->n_used + extra);
}

// hand over the particles that left each slab (one host read of the counts)
int migrate(pic_slabs *g) {
  for (int s = 0; s < g->S; ++s) {
    pic_ctx *c = g->ctx[s];
    if (c->n_used == 0 || (!c->G.open_lo && !c->G.open_hi)) continue;
    // only the particles of the two boundary rows can leave; the messages
    // start at a fraction of the slab and grow when a pass finds them full
    const bool fp32 = c->d.precision == PIC_FP32;
    int e = fp32 ? reserve_box32(g, c->n_used / 16 + 4096) : reserve_box(g, c->n_used / 16 + 4096);
    if (e) return e;
    for (;;) {
      const int64_t cap = fp32 ? g->box32_cap : g->box_cap;
      const unsigned blocks = (unsigned)((c->n_used + 255) / 256);
      PIC_CUDA(cudaMemsetAsync(g->d_box, 0, 2 * sizeof(long long), g->stream));
      if (fp32)
        ++c->launches, k_emigrate32<<<blocks, 256, 0, g->stream>>>(c->G, c->p32, c->n_used, g->box32[0], g->box32[1],
                                                                   cap, g->d_box);
      else
        ++c->launches, k_emigrate<<<blocks, 256, 0, g->stream>>>(c->G, c->p64, c->n_used, g->box[0], g->box[1], cap,
                                                                 g->d_box);
      PIC_CUDA(cudaMemcpyAsync(g->h_box, g->d_box, 2 * sizeof(long long), cudaMemcpyDeviceToHost, g->stream));
      PIC_CUDA(cudaStreamSynchronize(g->stream));
      const int64_t want = std::max(g->h_box[0], g->h_box[1]);
      for (int side = 0; side < 2; ++side) {
        const int64_t m = std::min<int64_t>(g->h_box[side], cap);
        if (m == 0) continue;
        pic_ctx *dst = g->ctx[s + (side ? 1 : -1)];
        if ((e = room(dst, m))) return e;
        const unsigned mb = (unsigned)((m + 255) / 256);
        if (fp32)
          ++dst->launches, k_immigrate32<<<mb, 256, 0, g->stream>>>(dst->p32, dst->n_used, g->box32[side], m);
        else
          ++dst->launches, k_immigrate<<<mb, 256, 0, g->stream>>>(dst->p64, dst->n_used, g->box[side], m);
        dst->n_used += m;
      }
      if (want <= cap) break;
      PIC_CUDA(cudaStreamSynchronize(g->stream));  // the messages are read before they are reallocated
      if ((e = fp32 ? reserve_box32(g, want) : reserve_box(g, want))) return e;
    }
  }
  PIC_CUDA(cudaGetLastError());
  return PIC_OK;
}

// node charge of every slab deposited, summed across interfaces and filtered
// as the current is (App. B), then the Gauss law over each slab's own
// interior rows (nodes 1 <= i <= nr - absorb_cells - 1 of the whole grid)
int slab_gauss(pic_slabs *g, bool snapshot, double *gmax, double *qmax) {
  for (pic_ctx *c : g->ctx) {
    cudaMemsetAsync(c->Q, 0, c->grid_elems * sizeof(double), g->stream);
    cudaMemsetAsync(c->Qa, 0, c->grid_elems * sizeof(double), g->stream);
    if (c->d.precision == PIC_FP32) charge32(c, c->Q, c->Qa);
    else charge64(c, c->Q, c->Qa);
  }
  for (int s = 0; s + 1 < g->S; ++s) {
    int e;
    if ((e = halo_sum(g, g->ctx[s], g->ctx[s + 1], g->ctx[s]->Q, g->ctx[s + 1]->Q)) ||
        (e = halo_sum(g, g->ctx[s], g->ctx[s + 1], g->ctx[s]->Qa, g->ctx[s + 1]->Qa)))
      return e;
  }
  const int L = g->d.absorb_profile == PIC_ABSORB_NONE ? 0 : g->d.absorb_cells;
  const int top = g->d.nr - L - 1;  // last interior node row of the whole grid
  *gmax = 0.0;
  *qmax = 0.0;
  for (int s = 0; s < g->S; ++s) {
    pic_ctx *c = g->ctx[s];
    filter_array(c, c->Q, c->Qt, 0, +1, g->d.n_filt);
    cudaMemsetAsync(c->d_cnt + CNT_GMAX, 0, 2 * sizeof(long long), g->stream);
    const int ilo = std::max(1 - c->G.i0, 0);
    const int ihi = std::min(top - c->G.i0, c->G.open_hi ? c->G.nr - 1 : c->G.nr);
    gauss_rows(c, ilo, ihi, snapshot);
    long long v[2];
    PIC_CUDA(cudaMemcpyAsync(v, c->d_cnt + CNT_GMAX, sizeof v, cudaMemcpyDeviceToHost, g->stream));
    PIC_CUDA(cudaStreamSynchronize(g->stream));
    double a, b;
    memcpy(&a, &v[0], sizeof a);
    memcpy(&b, &v[1], sizeof b);
    *gmax = std::max(*gmax, a);
    *qmax = std::max(*qmax, b);
  }
  return PIC_OK;
}

// one time step of the whole grid
int slab_step(pic_slabs *g) {
  const int S = g->S;
  const double t = g->step * g->d.dt;
  int e;
  if (g->d.precision == PIC_FP32) {
    // exact int64 sums across the interfaces, then the conversion
    for (pic_ctx *c : g->ctx) particles32(c, t);
    for (int s = 0; s + 1 < S; ++s)
      for (int k = 0; k < 3; ++k)
        if ((e = halo_sum(g, g->ctx[s], g->ctx[s + 1], g->ctx[s]->acc[k], g->ctx[s + 1]->acc[k]))) return e;
    for (pic_ctx *c : g->ctx) flux_from_acc(c);
  } else {
    for (pic_ctx *c : g->ctx) {
      for (int k = 0; k < 3; ++k) cudaMemsetAsync(c->F[k], 0, c->grid_elems * sizeof(double), g->stream);
      particles64(c, t);
    }
    for (int s = 0; s + 1 < S; ++s)
      for (int k = 0; k < 3; ++k)
        if ((e = halo_sum(g, g->ctx[s], g->ctx[s + 1], g->ctx[s]->F[k], g->ctx[s + 1]->F[k]))) return e;
  }
  if (g->d.n_filt > 0)
    for (pic_ctx *c : g->ctx) fields_filter(c);
  static const int B3[3] = {BR, BTH, BPH}, E3[3] = {ER, ETH, EPH}, ALL[6] = {ER, ETH, EPH, BR, BTH, BPH};
  for (pic_ctx *c : g->ctx) fields_b_half(c);
  if ((e = exchange_fields(g, B3, 3))) return e;
  for (pic_ctx *c : g->ctx) fields_e_full(c);
  if ((e = exchange_fields(g, E3, 3))) return e;
  for (pic_ctx *c : g->ctx) fields_b_half(c);
  for (pic_ctx *c : g->ctx) fields_finish(c);
  if ((e = exchange_fields(g, ALL, 6))) return e;
  if (g->d.precision == PIC_FP32)  // the gather copies again, now with the neighbours' rows
    for (pic_ctx *c : g->ctx) fields_copy32(c);
  g->step += 1;
  for (pic_ctx *c : g->ctx) c->step = g->step;
  pic_ctx *c0 = g->ctx[0];
  if (g->d.inject) {
    const int64_t slots = (int64_t)2 * g->d.pairs_per_cell * g->d.nth;
    if ((e = room(c0, slots))) return e;
    c0->next_id = g->next_id;
    inject(c0, g->step * g->d.dt);
    g->next_id = c0->next_id;
  }
  if ((e = migrate(g))) return e;
  for (pic_ctx *c : g->ctx) {
    c->steps_since_sort += 1;
    if (c->steps_since_sort >= g->d.sort_interval && (e = pic_compact(c))) return e;
  }
  return PIC_OK;
}

int group_status(pic_slabs *g) {
  for (pic_ctx *c : g->ctx) {
    const int e = pic_latch_status(c);
    if (e) return e;
  }
  return PIC_OK;
}

}  // namespace

extern "C" int pic_slabs_init(pic_slabs **out, const pic_desc *dd, int32_t nslabs, const int32_t *rows,
                              void *stream) {
  if (!out || !dd) return pic_fail(PIC_EINVAL, "null argument");
  *out = nullptr;
  pic_desc d = *dd;
  int e = pic_desc_defaults(&d);
  if (e) return e;
  if (nslabs < 1 || nslabs > d.nr) return pic_fail(PIC_EINVAL, "nslabs must be in [1, nr]");
  const int g = d.n_filt + 2;
  std::vector<int> a(nslabs + 1);
  for (int s = 0; s <= nslabs; ++s) a[s] = rows ? rows[s] : (int)((int64_t)d.nr * s / nslabs);
  if (a[0] != 0 || a[nslabs] != d.nr) return pic_fail(PIC_EINVAL, "slab rows must run from 0 to nr");
  for (int s = 0; s < nslabs; ++s)
    if (a[s + 1] - a[s] < 2 * g + 2)
      return pic_fail(PIC_EINVAL, "every slab needs at least 2 (n_filt + 2) + 2 rows (its halos)");
  const int L = d.absorb_profile == PIC_ABSORB_NONE ? 0 : d.absorb_cells;
  if (L + 1 > a[nslabs] - a[nslabs - 1]) return pic_fail(PIC_EINVAL, "the lossy layer must lie in the last slab");
  if (!(d.dt > 0.0)) {  // the whole grid's Courant step, shared by every slab
    pic_ctx *tmp = nullptr;
    pic_desc one = d;
    if ((e = pic_create_context(&tmp, one, stream, 0, d.nr, 0, 0))) return e;
    d.dt = tmp->G.dt;
    pic_destroy(tmp);
  }
  pic_slabs *G = new pic_slabs();
  G->d = d;
  G->S = nslabs;
  G->a = a;
  G->stream = (cudaStream_t)stream;
  for (int s = 0; s < nslabs; ++s) {
    pic_desc ds = d;
    ds.nr = a[s + 1] - a[s];
    if (s > 0) ds.inject = PIC_INJECT_OFF;  // the surface is in the first slab
    if (s + 1 < nslabs) ds.absorb_profile = PIC_ABSORB_NONE;  // the layer is in the last
    ds.capacity = 0;
    pic_ctx *c = nullptr;
    if ((e = pic_create_context(&c, ds, stream, a[s], d.nr, s > 0, s + 1 < nslabs))) {
      pic_slabs_destroy(G);
      return e;
    }
    c->have_snap = true;  // the group takes the Gauss snapshot over all slabs
    G->ctx.push_back(c);
  }
  // one fixed-point quantum for the whole grid: every slab raises and reads
  // the first slab's exponent, so the int64 sums of neighbours add exactly
  for (int s = 1; s < nslabs; ++s) G->ctx[s]->qexp = G->ctx[0]->qexp;
  G->stage_elems = (size_t)(g + 1) * G->ctx[0]->G.LD;
  if (cudaMalloc((void **)&G->stage, G->stage_elems * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void **)&G->d_box, 2 * sizeof(long long)) != cudaSuccess ||
      cudaMallocHost((void **)&G->h_box, 2 * sizeof(long long)) != cudaSuccess) {
    pic_slabs_destroy(G);
    return pic_fail(PIC_ENOMEM, "slab buffers");
  }
  *out = G;
  return PIC_OK;
}

extern "C" int pic_slabs_load_particles(pic_slabs *g, int64_t n, const double *x1, const double *x2,
                                        const double *u_r, const double *u_th, const double *u_ph, const double *qw,
                                        int32_t mem) {
  if (!g) return pic_fail(PIC_EINVAL, "null slab group");
  if (n < 0) return pic_fail(PIC_EINVAL, "n < 0");
  if (n == 0) return PIC_OK;
  if (!x1 || !x2 || !u_r || !u_th || !u_ph || !qw) return pic_fail(PIC_EINVAL, "null particle array");
  const double *src[6] = {x1, x2, u_r, u_th, u_ph, qw};
  const double *dv[6];
  double *stage = nullptr;
  if (mem == PIC_MEM_DEVICE) {
    for (int k = 0; k < 6; ++k) dv[k] = src[k];
  } else {
    PIC_CUDA(cudaMalloc((void **)&stage, 6 * (size_t)n * sizeof(double)));
    for (int k = 0; k < 6; ++k) {
      cudaMemcpyAsync(stage + (size_t)k * n, src[k], n * sizeof(double), cudaMemcpyHostToDevice, g->stream);
      dv[k] = stage + (size_t)k * n;
    }
  }
  int e = PIC_OK;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  const bool fp32 = g->d.precision == PIC_FP32;
  for (pic_ctx *c : g->ctx) {
    // count this slab's share, make room, append it
    cudaMemsetAsync(g->d_box, 0, sizeof(long long), g->stream);
    if (fp32)
      ++c->launches, k_load_slab32<<<blocks, 256, 0, g->stream>>>(c->G, Parts32{}, 0, n, dv[0], dv[1], dv[2], dv[3],
                                                                  dv[4], dv[5], g->next_id, g->d_box, c->d_err,
                                                                  c->qexp);
    else
      ++c->launches, k_load_slab<<<blocks, 256, 0, g->stream>>>(c->G, Parts64{}, 0, n, dv[0], dv[1], dv[2], dv[3],
                                                                dv[4], dv[5], g->next_id, g->d_box, c->d_err);
    cudaMemcpyAsync(g->h_box, g->d_box, sizeof(long long), cudaMemcpyDeviceToHost, g->stream);
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) { e = pic_fail(PIC_ECUDA, "slab load"); break; }
    const int64_t m = g->h_box[0];
    const int64_t slots = c->d.inject ? (int64_t)2 * c->d.pairs_per_cell * c->d.nth * (c->d.sort_interval + 2) : 0;
    if ((e = pic_reserve(c, c->n_used + 2 * m + slots + 1024))) break;
    cudaMemsetAsync(g->d_box, 0, sizeof(long long), g->stream);
    if (fp32)
      ++c->launches, k_load_slab32<<<blocks, 256, 0, g->stream>>>(c->G, c->p32, c->n_used, n, dv[0], dv[1], dv[2],
                                                                  dv[3], dv[4], dv[5], g->next_id, g->d_box, c->d_err,
                                                                  c->qexp);
    else
      ++c->launches, k_load_slab<<<blocks, 256, 0, g->stream>>>(c->G, c->p64, c->n_used, n, dv[0], dv[1], dv[2],
                                                                dv[3], dv[4], dv[5], g->next_id, g->d_box, c->d_err);
    c->n_used += m;
    c->need_sort = true;
    c->mix_sort = true;
  }
  cudaStreamSynchronize(g->stream);
  cudaFree(stage);
  if (e) return e;
  PIC_CUDA(cudaGetLastError());
  g->next_id += n;
  int he = 0;
  PIC_CUDA(cudaMemcpy(&he, g->ctx[0]->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (he & ERR_RANGE) {
    cudaMemset(g->ctx[0]->d_err, 0, sizeof(int));
    return pic_fail(PIC_EINVAL, "particle outside the grid, zero charge or non-finite momentum (dropped)");
  }
  g->have_snap = false;
  return PIC_OK;
}

extern "C" int pic_slabs_step(pic_slabs *g, int32_t nsteps) {
  if (!g) return pic_fail(PIC_EINVAL, "null slab group");
  if (nsteps < 0) return pic_fail(PIC_EINVAL, "nsteps < 0");
  int e;
  for (pic_ctx *c : g->ctx)  // FP32: bin the particles of a new load before stepping
    if (c->need_sort) {
      if ((e = pic_compact(c))) return e;
      c->need_sort = false;
    }
  if (!g->have_snap) {
    double a, b;
    if ((e = slab_gauss(g, true, &a, &b))) return e;
    g->have_snap = true;
  }
  for (int k = 0; k < nsteps; ++k)
    if ((e = slab_step(g))) return e;
  PIC_CUDA(cudaGetLastError());
  return group_status(g);
}

extern "C" int pic_slabs_get_fields(pic_slabs *g, int32_t which, double *out6, int64_t *n, int32_t mem) {
  if (!g || !n) return pic_fail(PIC_EINVAL, "null argument");
  const int rows = g->d.nr + 1, cols = g->d.nth + 1;
  const size_t plane = (size_t)rows * cols;
  *n = (int64_t)(6 * plane);
  if (!out6) return PIC_OK;
  const cudaMemcpyKind kind = mem == PIC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  int e = PIC_OK;
  for (int s = 0; s < g->S && !e; ++s) {
    pic_ctx *c = g->ctx[s];
    const int lr = c->d.nr + 1;
    double *tmp;
    PIC_CUDA(cudaMalloc((void **)&tmp, 6 * (size_t)lr * cols * sizeof(double)));
    int64_t m = 0;
    e = pic_get_fields(c, which, tmp, &m, PIC_MEM_DEVICE);
    // own node rows: [0, n_s), the last slab also its outer row
    const int own = s + 1 < g->S ? c->d.nr : c->d.nr + 1;
    for (int k = 0; k < 6 && !e; ++k)
      if (cudaMemcpyAsync(out6 + k * plane + (size_t)g->a[s] * cols, tmp + (size_t)k * lr * cols,
                          (size_t)own * cols * sizeof(double), kind, g->stream) != cudaSuccess)
        e = pic_fail(PIC_ECUDA, "slab field copy");
    cudaStreamSynchronize(g->stream);
    cudaFree(tmp);
  }
  return e ? e : group_status(g);
}

extern "C" int pic_slabs_get_flux(pic_slabs *g, double *out3, int64_t *n, int32_t mem) {
  if (!g || !n) return pic_fail(PIC_EINVAL, "null argument");
  const int gg = g->d.n_filt + 2, rows = g->d.nr + 2 * gg + 1, cols = g->d.nth + 1;
  const size_t plane = (size_t)rows * cols;
  *n = (int64_t)(3 * plane);
  if (!out3) return PIC_OK;
  const cudaMemcpyKind kind = mem == PIC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  int e = PIC_OK;
  for (int s = 0; s < g->S && !e; ++s) {
    pic_ctx *c = g->ctx[s];
    const int lr = c->d.nr + 2 * gg + 1;
    double *tmp;
    PIC_CUDA(cudaMalloc((void **)&tmp, 3 * (size_t)lr * cols * sizeof(double)));
    int64_t m = 0;
    e = pic_get_flux(c, tmp, &m, PIC_MEM_DEVICE);
    // own rows: the first slab from -g, the last up to nr + g (local plane row i + g)
    const int first = s == 0 ? -gg : 0, last = s + 1 < g->S ? c->d.nr - 1 : c->d.nr + gg;
    for (int k = 0; k < 3 && !e; ++k)
      if (cudaMemcpyAsync(out3 + k * plane + (size_t)(g->a[s] + first + gg) * cols,
                          tmp + (size_t)k * lr * cols + (size_t)(first + gg) * cols,
                          (size_t)(last - first + 1) * cols * sizeof(double), kind, g->stream) != cudaSuccess)
        e = pic_fail(PIC_ECUDA, "slab flux copy");
    cudaStreamSynchronize(g->stream);
    cudaFree(tmp);
  }
  return e;
}

extern "C" int pic_slabs_get_particles(pic_slabs *g, int64_t *n, double *x1, double *x2, double *u_r,
                                       double *u_th, double *u_ph, double *qw, int64_t *id, int32_t mem) {
  if (!g || !n) return pic_fail(PIC_EINVAL, "null argument");
  int64_t total = 0;
  std::vector<int64_t> cnt(g->S);
  int e;
  for (int s = 0; s < g->S; ++s) {
    if ((e = pic_get_particles(g->ctx[s], &cnt[s], nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                               mem)))
      return e;
    total += cnt[s];
  }
  if (!x1) { *n = total; return PIC_OK; }
  if (*n < total) { *n = total; return pic_fail(PIC_EINVAL, "output buffers too small"); }
  if (!x2 || !u_r || !u_th || !u_ph || !qw) return pic_fail(PIC_EINVAL, "null output array");
  int64_t off = 0;
  for (int s = 0; s < g->S; ++s) {
    int64_t m = cnt[s];
    if ((e = pic_get_particles(g->ctx[s], &m, x1 + off, x2 + off, u_r + off, u_th + off, u_ph + off, qw + off,
                               id ? id + off : nullptr, mem)))
      return e;
    off += m;
  }
  *n = off;
  return PIC_OK;
}

extern "C" int pic_slabs_get_moments(pic_slabs *g, pic_moments *out) {
  if (!g || !out) return pic_fail(PIC_EINVAL, "null argument");
  memset(out, 0, sizeof *out);
  int e;
  for (int s = 0; s < g->S; ++s) {
    pic_ctx *c = g->ctx[s];
    cudaMemsetAsync(c->d_acc, 0, ACC_N * sizeof(double), g->stream);
    cudaMemsetAsync(c->d_cnt + CNT_LIVE, 0, sizeof(long long), g->stream);
    field_energy_rows(c, c->G.open_hi ? c->G.nr - 1 : c->G.nr);
    if (c->d.precision == PIC_FP32) reduce_particles32(c);
    else reduce_particles64(c);
    long long cnt[CNT_N];
    double acc[ACC_N];
    PIC_CUDA(cudaMemcpyAsync(cnt, c->d_cnt, sizeof cnt, cudaMemcpyDeviceToHost, g->stream));
    PIC_CUDA(cudaMemcpyAsync(acc, c->d_acc, sizeof acc, cudaMemcpyDeviceToHost, g->stream));
    PIC_CUDA(cudaStreamSynchronize(g->stream));
    out->live += cnt[CNT_LIVE];
    out->deleted += cnt[CNT_DELETED];
    out->injected += cnt[CNT_INJECTED];
    out->inject_capped += cnt[CNT_CAPPED];
    out->axis_ties += cnt[CNT_TIES];
    out->kinetic_energy += acc[ACC_KIN];
    out->field_energy += acc[ACC_FIELD];
    out->total_charge += acc[ACC_CHARGE];
  }
  out->step = g->step;
  out->dt = g->d.dt;
  out->time = g->step * g->d.dt;
  double gm = 0.0, qm = 0.0;
  if (!g->have_snap) {
    out->gauss_residual = -1.0;
  } else {
    if ((e = slab_gauss(g, false, &gm, &qm))) return e;
    out->gauss_residual = qm > 0 ? gm / qm : gm;
  }
  return group_status(g);
}

extern "C" int pic_slabs_destroy(pic_slabs *g) {
  if (!g) return PIC_OK;
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (pic_ctx *c : g->ctx) pic_destroy(c);
  free_box(g);
  cudaFree(g->stage);
  cudaFree(g->d_box);
  if (g->h_box) cudaFreeHost(g->h_box);
  delete g;
  return PIC_OK;
}

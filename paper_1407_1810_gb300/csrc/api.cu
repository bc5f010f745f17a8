// api.cu -- the C-ABI of include/picsar.h: context set-up, the metric tables,
// particle loading, the step sequence and the getters.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pic_internal.h"

using namespace pic;

static thread_local std::string g_last_error;

int pic_fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

int pic_cuda_check(cudaError_t e, const char *what) {
  return pic_fail(e == cudaErrorMemoryAllocation ? PIC_ENOMEM : PIC_ECUDA,
                  std::string(what) + ": " + cudaGetErrorString(e));
}

extern "C" const char *pic_last_error(void) { return g_last_error.c_str(); }

extern "C" void pic_struct_sizes(int64_t *desc_bytes, int64_t *moments_bytes) {
  if (desc_bytes) *desc_bytes = (int64_t)sizeof(pic_desc);
  if (moments_bytes) *moments_bytes = (int64_t)sizeof(pic_moments);
}

namespace {

// ---- host copies of the stretching functions (Sec. 3.2) ----------------------
double h_fr(const pic_desc &d, double dxi, double x) {
  return d.r_map == PIC_R_LOG ? d.r_min * std::exp(x * dxi) : d.r_min + x * dxi;
}
double h_fth(const pic_desc &d, double x) {
  if (x < 0) x = 0;
  if (x > d.nth) x = d.nth;
  return d.th_map == PIC_TH_EQUAL_AREA ? std::acos(1.0 - 2.0 * x / d.nth) : M_PI * x / d.nth;
}

// rho: global radial grid coordinate; nr: the global row count
double sigma_star(const pic_desc &d, double rho, int nr) {
  const int L = d.absorb_cells;
  if (d.absorb_profile == PIC_ABSORB_NONE || L <= 0) return 0.0;
  double x = rho - (nr - L);
  if (x <= 0.0) return 0.0;
  double u = x / L;
  if (d.absorb_profile == PIC_ABSORB_QUADRATIC) return (d.absorb_sigma_max > 0 ? d.absorb_sigma_max : 3.0 / L) * u * u;
  return (d.absorb_sigma_max > 0 ? d.absorb_sigma_max : 2.0 / L) * u;
}

int check_desc(const pic_desc &d) {
  if (d.nr < 2 || d.nth < 2 || d.nth > 32000 || d.nr > 32000) return pic_fail(PIC_EINVAL, "nr, nth must be in [2, 32000]");
  if (!(d.r_min > 0.0) || !(d.r_max > d.r_min)) return pic_fail(PIC_EINVAL, "need 0 < r_min < r_max");
  if (d.r_map != PIC_R_LINEAR && d.r_map != PIC_R_LOG) return pic_fail(PIC_EINVAL, "bad r_map");
  if (d.th_map != PIC_TH_LINEAR && d.th_map != PIC_TH_EQUAL_AREA) return pic_fail(PIC_EINVAL, "bad th_map");
  if (d.n_filt < 0 || d.n_filt > 16) return pic_fail(PIC_EINVAL, "n_filt must be in [0, 16]");
  if (d.absorb_profile < 0 || d.absorb_profile > 2 || d.absorb_cells < 0 || d.absorb_cells >= d.nr)
    return pic_fail(PIC_EINVAL, "bad absorbing layer");
  if (d.vacuum < 0 || d.vacuum > 5) return pic_fail(PIC_EINVAL, "bad vacuum field kind");
  if (d.precision != PIC_FP64 && d.precision != PIC_FP32) return pic_fail(PIC_EINVAL, "bad precision");
  if (d.pusher != PIC_VAY && d.pusher != PIC_BORIS) return pic_fail(PIC_EINVAL, "bad pusher");
  if (d.inject < PIC_INJECT_OFF || d.inject > PIC_INJECT_VARIABLE) return pic_fail(PIC_EINVAL, "bad inject mode");
  if (d.inject && (d.pairs_per_cell < 1 || !(d.f_inj > 0.0) || d.f_inj > 1.0))
    return pic_fail(PIC_EINVAL, "injection needs pairs_per_cell >= 1 and 0 < f_inj <= 1");
  if (d.inject == PIC_INJECT_VARIABLE && !(d.inject_q > 0.0 && std::isfinite(d.inject_q)))
    return pic_fail(PIC_EINVAL, "variable-count injection needs a finite inject_q > 0");
  if (d.inject_smooth < 0 || d.inject_smooth > 64) return pic_fail(PIC_EINVAL, "inject_smooth must be in [0, 64]");
  if (d.r_map == PIC_R_LINEAR) {
    double dr = (d.r_max - d.r_min) / d.nr;
    if (d.r_min - (d.n_filt + 2) * dr <= 0.0)
      return pic_fail(PIC_EINVAL, "linear r map: the ghost cells inside the inner conductor reach r <= 0");
  }
  if (d.tile_shape < 0 || d.tile_shape > 2) return pic_fail(PIC_EINVAL, "tile_shape must be 0, 1 or 2");
  if (!(d.flux_quantum >= 0.0) || !std::isfinite(d.flux_quantum))
    return pic_fail(PIC_EINVAL, "flux_quantum must be finite and >= 0");
  if (d.precision == PIC_FP32 && d.nr + 2 * (d.n_filt + 2) >= 65536 - 2 * CELL_BIAS)
    return pic_fail(PIC_EINVAL, "FP32 path: grid too large for the packed cell index");
  return PIC_OK;
}

double courant_dt(const pic_desc &d, double dxi) {
  double m = 1e300;
  for (int i = 0; i < d.nr; ++i) {
    double ra = h_fr(d, dxi, i), rb = h_fr(d, dxi, i + 1);
    for (int j = 0; j < d.nth; ++j) {
      double v = std::fmin(rb - ra, ra * (h_fth(d, j + 1) - h_fth(d, j)));
      if (v < m) m = v;
    }
  }
  return d.courant * m;
}

template <typename T>
int dalloc(T **p, size_t n) {
  PIC_CUDA(cudaMalloc((void **)p, n * sizeof(T)));
  return PIC_OK;
}

// ---- metric tables ----------------------------------------------------------
int build_metric(pic_ctx *c) {
  const pic_desc &d = c->d;
  Grid &G = c->G;
  const int NRr = d.nr + 2 * G.PI + 1, NC = G.LD;
  const int nrg = G.nr_glob;  // rows of the whole grid (a slab's tables hold its global rows)
  // row tables 0-12 (geometry) and 13-20 (update coefficients); column
  // tables 0-11 and 17 (geometry) and 12-16 (update coefficients)
  const int nrow = 21, ncol = 18;
  const double hh = 0.5 * G.dt, dt = G.dt;
  std::vector<double> h((size_t)nrow * NRr + (size_t)ncol * NC, 0.0);
  auto row = [&](int t) { return h.data() + (size_t)t * NRr; };
  auto col = [&](int t) { return h.data() + (size_t)nrow * NRr + (size_t)t * NC; };
  const double dxi = G.dxi;
  auto fr = [&](double x) { return h_fr(d, dxi, x); };
  for (int ii = 0; ii < NRr; ++ii) {
    const int i = ii - G.PI + G.i0;  // global row
    double rn = fr(i), rn1 = fr(i + 1), rh = fr(i + 0.5), rhm = fr(i - 0.5);
    row(0)[ii] = rn;
    row(1)[ii] = rh;
    row(2)[ii] = 1.0 / rn;
    row(3)[ii] = 2.0 / (rn1 * rn1 - rn * rn);
    row(4)[ii] = rn1 - rn;
    row(5)[ii] = 1.0 / rh;
    row(6)[ii] = 1.0 / (2.0 * M_PI * rh * rh);
    row(7)[ii] = 2.0 / (rh * rh - rhm * rhm);
    row(8)[ii] = rh - rhm;
    row(9)[ii] = 1.0 - sigma_star(d, i, nrg);
    row(10)[ii] = 1.0 - sigma_star(d, i + 0.5, nrg);
    const double id2n = 2.0 / (rn1 * rn1 - rn * rn), id2h = 2.0 / (rh * rh - rhm * rhm);
    row(13)[ii] = hh / rn;
    row(14)[ii] = hh * id2n * rn;
    row(15)[ii] = hh * id2n * rn1;
    row(16)[ii] = hh * id2n * (rn1 - rn);
    row(17)[ii] = dt / rh;
    row(18)[ii] = dt * id2h * rhm;
    row(19)[ii] = dt * id2h * rh;
    row(20)[ii] = dt * id2h * (rh - rhm);
    if (i >= 0 && i <= nrg) {
      double a = std::fmax(i - 0.5, 0.0), b = std::fmin(i + 0.5, (double)nrg);
      row(11)[ii] = 2.0 * M_PI / 3.0 * (std::pow(fr(b), 3) - std::pow(fr(a), 3));
      row(12)[ii] = i < nrg ? 2.0 * M_PI / 3.0 * (std::pow(rn1, 3) - std::pow(rn, 3)) : 0.0;
    }
  }
  auto th = [&](double x) { return h_fth(d, x); };
  auto ctb = [&](int j) { return j < 0 ? 1.0 : (j >= d.nth ? -1.0 : std::cos(th(j + 0.5))); };
  for (int cc = 0; cc < NC; ++cc) {
    const int j = cc - G.PJ;
    if (j >= 0 && j <= d.nth) {
      col(0)[cc] = std::sin(th(j));
      col(1)[cc] = std::cos(th(j));
      col(9)[cc] = 1.0 / (ctb(j - 1) - ctb(j));
      col(10)[cc] = std::cos(th(std::fmax(j - 0.5, 0.0))) - std::cos(th(std::fmin(j + 0.5, (double)d.nth)));
    }
    if (j >= 0 && j < d.nth) {
      col(2)[cc] = 1.0 / (std::cos(th(j)) - std::cos(th(j + 1)));
      col(3)[cc] = 1.0 / (th(j + 1) - th(j));
      col(4)[cc] = std::sin(th(j + 0.5));
      col(5)[cc] = 1.0 / std::sin(th(j + 0.5));
      col(11)[cc] = std::cos(th(j)) - std::cos(th(j + 1));
      col(17)[cc] = std::cos(th(j + 0.5));
    }
    if (j >= 1 && j < d.nth) col(6)[cc] = 1.0 / (th(j + 0.5) - th(j - 0.5));
  }
  for (int cc = 0; cc < NC; ++cc) {  // products of the geometry columns (zero where a factor is)
    const int j = cc - G.PJ;
    const double stb = j >= 0 && j < d.nth ? col(4)[cc] : 0.0, stbm = cc >= 1 && j >= 1 && j <= d.nth ? col(4)[cc - 1] : 0.0;
    if (j >= 0 && j < d.nth) {
      col(12)[cc] = col(0)[cc] * col(2)[cc];
      col(13)[cc] = col(0)[cc + 1] * col(2)[cc];
      col(16)[cc] = col(5)[cc] * (0.5 / M_PI);
    }
    if (j >= 0 && j <= d.nth) {
      col(14)[cc] = stb * col(9)[cc];
      col(15)[cc] = stbm * col(9)[cc];
    }
  }
  PIC_CUDA(cudaMalloc((void **)&c->metric_buf, h.size() * sizeof(double)));
  PIC_CUDA(cudaMemcpy(c->metric_buf, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
  const double *R = c->metric_buf, *C = c->metric_buf + (size_t)nrow * NRr;
  auto dr = [&](int t) { return R + (size_t)t * NRr; };
  auto dc = [&](int t) { return C + (size_t)t * NC; };
  Metric &m = G.m;
  m.r_n = dr(0); m.r_h = dr(1); m.inv_r_n = dr(2); m.inv_dr2_n = dr(3); m.dr_n = dr(4);
  m.inv_r_h = dr(5); m.inv_area_h = dr(6); m.inv_dr2_h = dr(7); m.dr_h = dr(8);
  m.keep_n = dr(9); m.keep_h = dr(10); m.vol_r_n = dr(11); m.vol_r_h = dr(12);
  m.sin_t = dc(0); m.cos_t = dc(1); m.inv_dcos_t = dc(2); m.inv_dth_t = dc(3);
  m.sin_tb = dc(4); m.inv_sin_tb = dc(5); m.inv_dtb = dc(6);
  m.inv_dcos_tb = dc(9); m.vol_t_n = dc(10); m.vol_t_h = dc(11);
  m.bR = dr(13); m.bT0 = dr(14); m.bT1 = dr(15); m.bP = dr(16);
  m.eR = dr(17); m.eT0 = dr(18); m.eT1 = dr(19); m.eP = dr(20);
  m.cB1 = dc(12); m.cB2 = dc(13); m.cE1 = dc(14); m.cE2 = dc(15); m.cF = dc(16);
  m.cos_tb = dc(17);
  return PIC_OK;
}

// ---- particle buffers ----------------------------------------------------------
void free_parts(pic_ctx *c) {
  Parts64 *a[2] = {&c->p64, &c->q64};
  for (Parts64 *p : a) {
    cudaFree(p->x1); cudaFree(p->x2); cudaFree(p->ur); cudaFree(p->ut); cudaFree(p->up); cudaFree(p->qw);
    cudaFree(p->id);
    *p = Parts64{};
  }
  Parts32 *b[2] = {&c->p32, &c->q32};
  for (Parts32 *p : b) {
    cudaFree(p->cell); cudaFree(p->dx); cudaFree(p->dy); cudaFree(p->ur); cudaFree(p->ut); cudaFree(p->up);
    cudaFree(p->qw); cudaFree(p->id);
    *p = Parts32{};
  }
  cudaFree(c->scratch);
  c->scratch = nullptr;
}

int alloc_parts(pic_ctx *c, int64_t cap) {
  const size_t n = (size_t)cap;
  if (c->d.precision == PIC_FP64) {
    Parts64 *a[2] = {&c->p64, &c->q64};
    for (Parts64 *p : a) {
      int e;
      if ((e = dalloc(&p->x1, n)) || (e = dalloc(&p->x2, n)) || (e = dalloc(&p->ur, n)) || (e = dalloc(&p->ut, n)) ||
          (e = dalloc(&p->up, n)) || (e = dalloc(&p->qw, n)) || (e = dalloc(&p->id, n)))
        return e;
    }
    PIC_CUDA(cudaMemset(c->p64.qw, 0, n * sizeof(double)));
  } else {
    Parts32 *a[2] = {&c->p32, &c->q32};
    for (Parts32 *p : a) {
      int e;
      if ((e = dalloc(&p->cell, n)) || (e = dalloc(&p->dx, n)) || (e = dalloc(&p->dy, n)) ||
          (e = dalloc(&p->ur, n)) || (e = dalloc(&p->ut, n)) || (e = dalloc(&p->up, n)) ||
          (e = dalloc(&p->qw, n)) || (e = dalloc(&p->id, n)))
        return e;
    }
    PIC_CUDA(cudaMemset(c->p32.qw, 0, n * sizeof(float)));
  }
  // scratch: block counts of the FP64 path's stable compaction
  c->scratch_bytes = ((size_t)cap / 256 + 2) * sizeof(long long);
  PIC_CUDA(cudaMalloc(&c->scratch, c->scratch_bytes));
  c->cap = cap;
  return PIC_OK;
}

// grow the particle buffers to new_cap keeping [0, n_used)
int grow_parts(pic_ctx *c, int64_t new_cap) {
  pic_ctx tmp;
  tmp.d = c->d;
  tmp.tiles = c->tiles;
  int e = alloc_parts(&tmp, new_cap);
  if (e) { free_parts(&tmp); return e; }
  const size_t n = (size_t)c->n_used;
  if (c->d.precision == PIC_FP64) {
    cudaMemcpyAsync(tmp.p64.x1, c->p64.x1, n * 8, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tmp.p64.x2, c->p64.x2, n * 8, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tmp.p64.ur, c->p64.ur, n * 8, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tmp.p64.ut, c->p64.ut, n * 8, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tmp.p64.up, c->p64.up, n * 8, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tmp.p64.qw, c->p64.qw, n * 8, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tmp.p64.id, c->p64.id, n * 8, cudaMemcpyDeviceToDevice, c->stream);
  } else {
    cudaMemcpyAsync(tmp.p32.cell, c->p32.cell, n * 4, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tmp.p32.dx, c->p32.dx, n * 4, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tmp.p32.dy, c->p32.dy, n * 4, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tmp.p32.ur, c->p32.ur, n * 4, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tmp.p32.ut, c->p32.ut, n * 4, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tmp.p32.up, c->p32.up, n * 4, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tmp.p32.qw, c->p32.qw, n * 4, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(tmp.p32.id, c->p32.id, n * 8, cudaMemcpyDeviceToDevice, c->stream);
  }
  PIC_CUDA(cudaStreamSynchronize(c->stream));
  free_parts(c);
  c->p64 = tmp.p64; c->q64 = tmp.q64; c->p32 = tmp.p32; c->q32 = tmp.q32;
  c->scratch = tmp.scratch; c->scratch_bytes = tmp.scratch_bytes;
  c->cap = new_cap;
  tmp.p64 = tmp.q64 = Parts64{};
  tmp.p32 = tmp.q32 = Parts32{};
  tmp.scratch = nullptr;
  return PIC_OK;
}

int64_t inject_slots(const pic_ctx *c) { return c->d.inject ? (int64_t)2 * c->d.pairs_per_cell * c->d.nth : 0; }

// ---- layout conversion between the padded arrays and the dense API planes ----
__global__ void k_pack(Grid G, const double *__restrict__ src, double *__restrict__ dst, int i_lo, int rows, int cols,
                       int imax, int jmax, int unpack) {
  const int j = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * 8 + threadIdx.y;
  if (r >= rows || j >= cols) return;
  const int i = i_lo + r;
  const size_t o = gidx(G, i, j), q = (size_t)r * cols + j;
  const bool in = i <= imax && j <= jmax;
  if (unpack) { if (in) ((double *)src)[o] = dst[q]; }
  else dst[q] = in ? src[o] : 0.0;
}

// plasma plus analytic field of component k at its staggered points, time t
__global__ void k_pack_total(Grid G, const double *__restrict__ src, double *__restrict__ dst, int k, int rows,
                             int cols, int imax, int jmax, double t) {
  const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
  if (i >= rows || j >= cols) return;
  const size_t q = (size_t)i * cols + j;
  if (i > imax || j > jmax) { dst[q] = 0.0; return; }
  const Metric &m = G.m;
  const double r = stag_i(k) ? m.r_h[i + G.PI] : m.r_n[i + G.PI];
  const double st = stag_j(k) ? m.sin_tb[j + G.PJ] : m.sin_t[j + G.PJ];
  const double ct = stag_j(k) ? m.cos_tb[j + G.PJ] : m.cos_t[j + G.PJ];
  double E[3], B[3];
  const Vac<double> V{G.vacuum, G.b0, G.r_min, omega_at(G.omega, G.t_spin, t)};
  vacuum_field<double>(V, r, st, ct, false, E, B);
  dst[q] = src[gidx(G, i, j)] + (k < 3 ? E[k] : B[k - 3]);
}

__global__ void k_grid_coords(Grid G, int64_t n, const double *__restrict__ r, const double *__restrict__ th,
                              double *x1, double *x2) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  x1[k] = map_r_inv(G, r[k]);
  x2[k] = map_th_inv(G, th[k]);
}

int to_user(pic_ctx *c, const double *dsrc, double *out, size_t n, int mem) {
  PIC_CUDA(cudaMemcpyAsync(out, dsrc, n * sizeof(double),
                           mem == PIC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  PIC_CUDA(cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

int latch_errors(pic_ctx *c) {
  int e = 0;
  PIC_CUDA(cudaMemcpyAsync(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  PIC_CUDA(cudaStreamSynchronize(c->stream));
  c->host_err |= e;
  return PIC_OK;
}

int status(pic_ctx *c) {
  const int e = c->host_err;
  if (e & ERR_NAN) return pic_fail(PIC_ENAN, "non-finite particle state");
  if (e & ERR_COURANT) return pic_fail(PIC_ECOURANT, "a particle crossed more than one grid line in one step");
  if (e & ERR_CAPACITY) return pic_fail(PIC_ECAPACITY, "particle buffer full");
  if (e & ERR_RANGE) return pic_fail(PIC_EINVAL, "particle outside the grid");
  if (e & ERR_TIMEOUT) return pic_fail(PIC_ETIMEOUT, "a bounded device-side wait gave up");
  return PIC_OK;
}

// ---- loading ---------------------------------------------------------------
__global__ void k_load64(Grid G, Parts64 P, int64_t base, int64_t n, const double *x1, const double *x2,
                         const double *ur, const double *ut, const double *up, const double *qw, int64_t id0,
                         int *err) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  // all six reads first, then the checks (without short-circuit): from
  // pinned host memory each dependent read would cost a host-link round trip
  const double a = x1[k], b = x2[k], q = qw[k], vr = ur[k], vt = ut[k], vp = up[k];
  const bool ok = (a >= -(double)(G.n_filt + 1)) & (a < (double)(G.nr_glob + G.n_filt + 1)) & (b >= 0.0) & (b <= G.nth) &
                  (q != 0.0) & isfinite(q) & isfinite(vr) & isfinite(vt) & isfinite(vp);
  const int64_t d = base + k;
  if (!ok) { atomicOr(err, ERR_RANGE); P.qw[d] = 0.0; return; }
  P.x1[d] = a; P.x2[d] = b; P.ur[d] = vr; P.ut[d] = vt; P.up[d] = vp; P.qw[d] = q; P.id[d] = id0 + k;
}

__global__ void k_load32(Grid G, Parts32 P, int64_t base, int64_t n, const double *x1, const double *x2,
                         const double *ur, const double *ut, const double *up, const double *qw, int64_t id0,
                         int *err, long long *qexp) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int qe = (int)QEXP_NONE;
  if (k < n) {
    // all six reads first, then the checks (without short-circuit): from
    // pinned host memory each dependent read would cost a host-link round trip
    const double a = x1[k], b = x2[k], q = qw[k], vr = ur[k], vt = ut[k], vp = up[k];
    const bool ok = (a >= -(double)(G.n_filt + 1)) & (a < (double)(G.nr_glob + G.n_filt + 1)) & (b >= 0.0) &
                    (b <= G.nth) & (fabs(q) >= 0x1p-100) & (fabs(q) <= 0x1p100) & isfinite(vr) & isfinite(vt) &
                    isfinite(vp);
    const int64_t d = base + k;
    if (!ok) {
      atomicOr(err, ERR_RANGE);
      P.qw[d] = 0.0;
    } else {
      // cell = floor(x); offset rounded to FP32 and kept in [0, 1)
      int ci = (int)floor(a), cj = (int)floor(b);
      if (cj > G.nth - 1) cj = G.nth - 1;
      float ox = (float)(a - ci), oy = (float)(b - cj);
      if (ox >= 1.0f) { ox = 0.0f; ++ci; }
      if (oy >= 1.0f && cj < G.nth - 1) { oy = 0.0f; ++cj; }
      P.cell[d] = ((uint32_t)(ci + CELL_BIAS) << 16) | (uint32_t)cj;  // whole-grid row
      P.dx[d] = ox; P.dy[d] = oy;
      P.ur[d] = (float)vr; P.ut[d] = (float)vt; P.up[d] = (float)vp; P.qw[d] = (float)q;
      P.id[d] = id0 + k;
      qe = charge_exp(fabsf((float)q));
    }
  }
  raise_qexp(qexp, qe);  // every lane of the warp reaches this
}

__global__ void k_export32(Parts32 P, int64_t n, double *x1, double *x2, double *ur, double *ut, double *up, double *qw,
                           int64_t *id) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t c = P.cell[k];
  x1[k] = (double)((int)(c >> 16) - CELL_BIAS) + (double)P.dx[k];
  x2[k] = (double)(c & 0xffffu) + (double)P.dy[k];
  ur[k] = P.ur[k]; ut[k] = P.ut[k]; up[k] = P.up[k]; qw[k] = P.qw[k];
  if (id) id[k] = P.id[k];
}

int compact(pic_ctx *c) {
  if (c->d.precision == PIC_FP64) compact64(c);
  else sort32(c);
  c->steps_since_sort = 0;
  return latch_errors(c);
}

// Profiling records a start/stop event pair per phase per step on the
// context's stream; the durations are summed when pic_get_profile reads them.
int prof_begin(pic_ctx *c, int slot) {
  if (!c->prof) return -1;
  if (c->ev_used + 2 > c->ev_pool.size()) {
    for (int k = 0; k < 64; ++k) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      c->ev_pool.push_back(e);
    }
    c->ev_slot.resize(c->ev_pool.size() / 2, 0);
  }
  const int pair = (int)(c->ev_used / 2);
  c->ev_slot[pair] = slot;
  cudaEventRecord(c->ev_pool[c->ev_used], c->stream);
  c->ev_used += 2;
  return pair;
}

void prof_end(pic_ctx *c, int pair) {
  if (pair < 0) return;
  cudaEventRecord(c->ev_pool[2 * (size_t)pair + 1], c->stream);
}

void prof_drain(pic_ctx *c) {
  if (c->ev_used == 0) return;
  cudaEventSynchronize(c->ev_pool[c->ev_used - 1]);
  for (size_t p = 0; p < c->ev_used / 2; ++p) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[2 * p], c->ev_pool[2 * p + 1]) == cudaSuccess) {
      c->prof_ms[c->ev_slot[p]] += ms;
      c->prof_launch[c->ev_slot[p]] += 1;
    }
  }
  c->ev_used = 0;
}

}  // namespace

// errors latched on the device, then the status they give (for the other
// translation units' entry points)
int pic_latch_status(pic_ctx *c) {
  int e = latch_errors(c);
  return e ? e : status(c);
}

int pic_grow_particles(pic_ctx *c, int64_t new_cap) { return grow_parts(c, new_cap); }
int pic_reserve(pic_ctx *c, int64_t need) {
  if (c->cap == 0) return alloc_parts(c, std::max<int64_t>(need, 1024));
  if (need > c->cap) return grow_parts(c, need * 3 / 2 + 1024);
  return PIC_OK;
}
int pic_compact(pic_ctx *c) { return compact(c); }

// =============================================================================
// tile geometry and cell bins of the FP32 path for a tile shape (0: 16 x 16,
// 1: 8 x 32, 2: 32 x 8 cells)
static int alloc_bins(pic_ctx *c, int shape) {
  Tiles &T = c->tiles;
  T.TI = shape == 1 ? 8 : (shape == 2 ? 32 : 16);
  T.TJ = shape == 1 ? 32 : (shape == 2 ? 8 : 16);
  T.tc = T.TI * T.TJ;
  T.nti = (c->d.nr + 2 * c->G.g + T.TI - 1) / T.TI;
  T.ntj = (c->d.nth + T.TJ - 1) / T.TJ;
  T.ntiles = T.nti * T.ntj;
  T.nbins = (int64_t)T.ntiles * T.tc + 1;
  const int64_t nblk = T.nbins / SCAN_CHUNK + 2;
  int e;
  if ((e = dalloc(&T.start, (size_t)T.nbins + 1)) || (e = dalloc(&T.cursor, (size_t)T.nbins + 1)) ||
      (e = dalloc(&T.bsum, 2 * (size_t)nblk)) || (e = dalloc(&T.ucount, (size_t)T.ntiles + 1)) ||
      (e = dalloc(&T.usum, 2 * ((size_t)T.ntiles / SCAN_CHUNK + 2))))
    return e;
  PIC_CUDA(cudaMemset(T.start, 0, (T.nbins + 1) * sizeof(int64_t)));
  return PIC_OK;
}

int pic_desc_defaults(pic_desc *d) {
  if (d->q_over_m == 0.0) d->q_over_m = 1.0;
  if (d->pairs_per_cell == 0) d->pairs_per_cell = 2;
  if (d->sort_interval <= 0) d->sort_interval = 20;
  return check_desc(*d);
}

// A context over rows [i0, i0 + d.nr) of a grid of nr_glob rows (the whole
// grid: i0 = 0, nr_glob = d.nr); d has been checked by pic_desc_defaults
// against the whole grid.
int pic_create_context(pic_ctx **out, const pic_desc &d, void *stream, int i0, int nr_glob, int open_lo,
                       int open_hi) {
  *out = nullptr;
  int e;
  pic_ctx *c = new pic_ctx();
  c->d = d;
  c->stream = (cudaStream_t)stream;
  cudaGetDevice(&c->device);
  Grid &G = c->G;
  G.nr = d.nr; G.nth = d.nth; G.n_filt = d.n_filt; G.g = d.n_filt + 2;
  G.i0 = i0; G.nr_glob = nr_glob; G.open_lo = open_lo; G.open_hi = open_hi;
  G.PI = G.g + PAD; G.PJ = PAD;
  G.LD = ((d.nth + 1 + 2 * G.PJ) + 7) / 8 * 8;
  G.r_map = d.r_map; G.th_map = d.th_map; G.r_min = d.r_min;
  G.dxi = d.r_map == PIC_R_LOG ? std::log(d.r_max / d.r_min) / nr_glob : (d.r_max - d.r_min) / nr_glob;
  G.dt = d.dt > 0.0 ? d.dt : courant_dt(d, G.dxi);
  if (!(G.dt > 0.0)) { delete c; return pic_fail(PIC_EINVAL, "dt must be > 0 (set dt or courant)"); }
  G.qm = d.q_over_m; G.vacuum = d.vacuum; G.pusher = d.pusher;
  G.b0 = d.b0; G.omega = d.omega; G.t_spin = d.t_spin;
  G.absorb_cells = d.absorb_profile == PIC_ABSORB_NONE ? 0 : d.absorb_cells;
  c->grid_elems = (size_t)(d.nr + 2 * G.PI + 1) * G.LD;
  const size_t ge = c->grid_elems;
  auto fail = [&](int code) { pic_destroy(c); return code; };
  if ((e = build_metric(c))) return fail(e);
  for (int k = 0; k < 6; ++k)
    if ((e = dalloc(&c->f[k], ge))) return fail(e);
  for (int k = 0; k < 3; ++k)
    if ((e = dalloc(&c->F[k], ge)) || (e = dalloc(&c->Ft[k], ge))) return fail(e);
  if ((e = dalloc(&c->Q, ge)) || (e = dalloc(&c->Qa, ge)) || (e = dalloc(&c->Qt, ge)) || (e = dalloc(&c->gsnap, ge)))
    return fail(e);
  for (int k = 0; k < 6; ++k) cudaMemset(c->f[k], 0, ge * 8);
  for (int k = 0; k < 3; ++k) { cudaMemset(c->F[k], 0, ge * 8); cudaMemset(c->Ft[k], 0, ge * 8); }
  cudaMemset(c->Q, 0, ge * 8); cudaMemset(c->Qa, 0, ge * 8); cudaMemset(c->Qt, 0, ge * 8);
  cudaMemset(c->gsnap, 0, ge * 8);
  if (d.precision == PIC_FP32) {
    for (int k = 0; k < 6; ++k) {
      if ((e = dalloc(&c->f32[k], ge))) return fail(e);
      cudaMemset(c->f32[k], 0, ge * 4);
    }
    for (int k = 0; k < 3; ++k) {
      if ((e = dalloc(&c->acc[k], ge))) return fail(e);
      cudaMemset(c->acc[k], 0, ge * 8);
    }
    {
      std::vector<float> rn(d.nr + 2 * G.PI + 1);
      // f_r of each padded row (global rows: a radial slab starts at row i0)
      for (size_t ii = 0; ii < rn.size(); ++ii) rn[ii] = (float)h_fr(d, G.dxi, (double)ii - G.PI + G.i0);
      // The grid bounds the arguments of the move's series: dx dxi <= dxi for
      // exp; with eps = dt / r(-g) (speed < c) the relative displacement s <=
      // 2 eps + 3 eps^2 for log1p and the turning angle below eps for atan and
      // the sin / cos series.  With dxi <= 1/16 and eps <= 1/40 every series'
      // relative truncation stays below 2^-28, 1/16 of an FP32 ulp (at the
      // bounds, evaluated in FP64: exp 8.8e-11, log1p 2.9e-9, atan and the
      // sin / cos series below 1e-13), so the step uses the series without
      // the general fallback
      c->small_steps = d.r_map == PIC_R_LOG && G.dxi <= 1.0 / 16 && G.dt / h_fr(d, G.dxi, -G.g) <= 1.0 / 40;
      if ((e = dalloc(&c->r_n32, rn.size()))) return fail(e);
      PIC_CUDA(cudaMemcpy(c->r_n32, rn.data(), rn.size() * sizeof(float), cudaMemcpyHostToDevice));
      // sine and cosine of the node angle pi j / nth of the linear theta map
      // per padded column, each the sine of an angle measured from the nearer
      // pole or from the equator (exact zeros and ones at the poles and the
      // equator), rounded once to FP32
      std::vector<float2> tn(G.LD);
      for (int jj = 0; jj < G.LD; ++jj) {
        const double j = (double)(jj - G.PJ), m = std::min(j, d.nth - j);
        tn[jj] = make_float2((float)std::sin(M_PI * m / d.nth), (float)std::sin(M_PI * (d.nth - 2.0 * j) / (2.0 * d.nth)));
      }
      if ((e = dalloc(&c->th_n32, tn.size()))) return fail(e);
      PIC_CUDA(cudaMemcpy(c->th_n32, tn.data(), tn.size() * sizeof(float2), cudaMemcpyHostToDevice));
    }
    c->tiles.row0 = -G.g;
    if ((e = alloc_bins(c, d.tile_shape))) return fail(e);
    if (tiles32_setup(c)) return fail(pic_fail(PIC_ECUDA, "tensor maps of the field window could not be encoded"));
  }
  if ((e = dalloc(&c->sig, 2 * ((size_t)d.nth + 1)))) return fail(e);
  if ((e = dalloc(&c->d_err, 1)) || (e = dalloc(&c->d_cnt, CNT_N)) || (e = dalloc(&c->d_acc, ACC_N))) return fail(e);
  cudaMemset(c->d_err, 0, sizeof(int));
  cudaMemset(c->d_cnt, 0, CNT_N * sizeof(long long));
  c->qexp = c->d_cnt + CNT_QEXP;
  {  // fixed-point exponent: raised on the device by the charges loaded or injected
    long long q0 = QEXP_NONE;
    if (d.flux_quantum > 0.0)
      q0 = std::min<long long>(QEXP_MAX, std::max<long long>(QEXP_MIN, (long long)std::ceil(std::log2(d.flux_quantum)) + KFIX));
    PIC_CUDA(cudaMemcpy(c->qexp, &q0, sizeof q0, cudaMemcpyHostToDevice));
  }
  if ((e = dalloc(&c->tie_step, TIE_LOG)) || (e = dalloc(&c->tie_id, TIE_LOG)) || (e = dalloc(&c->tie_sign, TIE_LOG)))
    return fail(e);
  PIC_CUDA(cudaMallocHost((void **)&c->h_pinned, 64));
  PIC_CUDA(cudaDeviceSynchronize());
  *out = c;
  return PIC_OK;
}

extern "C" int pic_init_grid(pic_ctx **out, const pic_desc *dd, void *stream) {
  if (!out || !dd) return pic_fail(PIC_EINVAL, "null argument");
  *out = nullptr;
  pic_desc d = *dd;
  int e = pic_desc_defaults(&d);
  if (e) return e;
  return pic_create_context(out, d, stream, 0, d.nr, 0, 0);
}

// Device-visible addresses of six host arrays that are page-locked (pinned):
// the load kernel then reads them in place -- on a Grace host over
// NVLink-C2C -- with no staging copy.  False for pageable memory.
static bool pinned_views(const double *const src[6], const double *dv[6]) {
  for (int k = 0; k < 6; ++k) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, src[k]) != cudaSuccess) {
      cudaGetLastError();  // clear the sticky-free error of the query
      return false;
    }
    if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return false;
    dv[k] = static_cast<const double *>(a.devicePointer);
  }
  return true;
}

extern "C" int pic_load_particles(pic_ctx *c, int64_t n, const double *x1, const double *x2, const double *u_r,
                                  const double *u_th, const double *u_ph, const double *qw, int32_t mem) {
  if (!c) return pic_fail(PIC_EINVAL, "null context");
  if (n < 0) return pic_fail(PIC_EINVAL, "n < 0");
  if (n == 0) return PIC_OK;
  if (!x1 || !x2 || !u_r || !u_th || !u_ph || !qw) return pic_fail(PIC_EINVAL, "null particle array");
  int e;
  const int64_t room = inject_slots(c) * (c->d.sort_interval + 2);
  if (c->cap == 0) {
    int64_t cap = c->d.capacity > 0 ? c->d.capacity : 2 * n + room + 1024;
    if (cap < n + room) cap = n + room;
    if ((e = alloc_parts(c, cap))) return e;
  } else if (c->n_used + n + room > c->cap) {
    if ((e = grow_parts(c, (c->n_used + n + room) * 3 / 2 + 1024))) return e;
  }
  // device views of the input: device arrays and pinned host arrays are read
  // in place, pageable host arrays are staged in chunks
  const double *const all[6] = {x1, x2, u_r, u_th, u_ph, qw};
  const double *pv[6];
  const bool direct = mem == PIC_MEM_DEVICE || pinned_views(all, pv);
  if (mem == PIC_MEM_DEVICE)
    for (int k = 0; k < 6; ++k) pv[k] = all[k];
  const int64_t chunk = direct ? n : ((int64_t)1 << 22);
  double *stage = nullptr;
  if (!direct) PIC_CUDA(cudaMalloc((void **)&stage, 6 * (size_t)chunk * sizeof(double)));
  for (int64_t off = 0; off < n; off += chunk) {
    const int64_t m = std::min(chunk, n - off);
    const double *src[6] = {x1 + off, x2 + off, u_r + off, u_th + off, u_ph + off, qw + off};
    const double *dv[6];
    for (int k = 0; k < 6; ++k) {
      if (direct) dv[k] = pv[k] + off;
      else {
        double *s = stage + (size_t)k * chunk;
        cudaMemcpyAsync(s, src[k], m * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        dv[k] = s;
      }
    }
    const unsigned blocks = (unsigned)((m + 255) / 256);
    if (c->d.precision == PIC_FP64)
      ++c->launches, k_load64<<<blocks, 256, 0, c->stream>>>(c->G, c->p64, c->n_used + off, m, dv[0], dv[1], dv[2], dv[3], dv[4],
                                             dv[5], c->next_id + off, c->d_err);
    else
      ++c->launches, k_load32<<<blocks, 256, 0, c->stream>>>(c->G, c->p32, c->n_used + off, m, dv[0], dv[1], dv[2], dv[3], dv[4],
                                             dv[5], c->next_id + off, c->d_err, c->qexp);
    if (!direct) PIC_CUDA(cudaStreamSynchronize(c->stream));
  }
  PIC_CUDA(cudaGetLastError());
  PIC_CUDA(cudaStreamSynchronize(c->stream));
  cudaFree(stage);
  int he = 0;
  PIC_CUDA(cudaMemcpy(&he, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  c->n_used += n;
  c->next_id += n;
  if (he & ERR_RANGE) {
    cudaMemset(c->d_err, 0, sizeof(int));
    return pic_fail(PIC_EINVAL, "particle outside the grid, zero charge or non-finite momentum (dropped)");
  }
  if (c->d.precision == PIC_FP32) {
    c->need_sort = true;  // binned by the next step (appended particles are valid unbinned)
    c->mix_sort = true;
  }
  return PIC_OK;
}

// One time step, enqueued on c->stream without any host synchronisation
// (also the unit the ensemble captures into a CUDA graph).
void pic_step_body(pic_ctx *c) {
  const double t = c->step * c->G.dt;
  int pr = prof_begin(c, PROF_PARTICLES);
  if (c->d.precision == PIC_FP64) {
    for (int k = 0; k < 3; ++k) cudaMemsetAsync(c->F[k], 0, c->grid_elems * 8, c->stream);
    particles64(c, t);
    prof_end(c, pr);
  } else {
    particles32(c, t);
    prof_end(c, pr);
    pr = prof_begin(c, PROF_REDUCE);
    flux_from_acc(c);
    prof_end(c, pr);
  }
  if (c->d.n_filt > 0) {
    pr = prof_begin(c, PROF_FILTER);
    fields_filter(c);
    prof_end(c, pr);
  }
  pr = prof_begin(c, PROF_FIELDS);
  fields_b_half(c);
  fields_e_full(c);
  fields_b_half(c);
  fields_finish(c);
  prof_end(c, pr);
  c->step += 1;
  if (c->d.inject) {
    pr = prof_begin(c, PROF_INJECT);
    inject(c, c->step * c->G.dt);
    prof_end(c, pr);
  }
  c->steps_since_sort += 1;
  if (c->prof) c->prof_steps += 1;
}

// Work that needs the host before steps can be enqueued blindly: a pending
// sort, the Gauss snapshot, and room for `steps` steps of injection.
int pic_prepare_steps(pic_ctx *c, int steps) {
  if (c->need_sort) {
    int e = compact(c);
    if (e) return e;
    c->need_sort = false;
  }
  if (!c->have_snap) moments(c, true, nullptr);
  const int64_t need = c->n_used + inject_slots(c) * (int64_t)steps;
  if (c->d.inject && need > c->cap) {
    int e = compact(c);
    if (e) return e;
    const int64_t need2 = c->n_used + inject_slots(c) * (int64_t)steps;
    if (need2 > c->cap && (e = grow_parts(c, need2 * 3 / 2 + 1024))) return e;
  }
  return PIC_OK;
}

extern "C" int pic_step(pic_ctx *c, int32_t nsteps) {
  if (!c) return pic_fail(PIC_EINVAL, "null context");
  if (nsteps < 0) return pic_fail(PIC_EINVAL, "nsteps < 0");
  int done = 0;
  while (done < nsteps) {
    // steps up to the next sort run without host synchronisation
    int block = std::min(nsteps - done, std::max(1, c->d.sort_interval - c->steps_since_sort));
    if (c->d.inject) block = std::min(block, 64);
    int e = pic_prepare_steps(c, block);
    if (e) return e;
    for (int s = 0; s < block; ++s) pic_step_body(c);
    done += block;
    if (c->steps_since_sort >= c->d.sort_interval) {
      int pr = prof_begin(c, PROF_SORT);
      e = compact(c);
      prof_end(c, pr);
      if (e) return e;
    }
    if (c->ev_used > 4096) prof_drain(c);
  }
  PIC_CUDA(cudaGetLastError());
  return status(c);
}

extern "C" int pic_get_fields(pic_ctx *c, int32_t which, double *out6, int64_t *n, int32_t mem) {
  if (!c || !n) return pic_fail(PIC_EINVAL, "null argument");
  if (which != PIC_FIELDS_PLASMA && which != PIC_FIELDS_TOTAL) return pic_fail(PIC_EINVAL, "bad field selector");
  const int rows = c->d.nr + 1, cols = c->d.nth + 1;
  const size_t plane = (size_t)rows * cols;
  *n = (int64_t)(6 * plane);
  if (!out6) return PIC_OK;
  double *tmp;
  PIC_CUDA(cudaMalloc((void **)&tmp, 6 * plane * sizeof(double)));
  dim3 gr((cols + 31) / 32, (rows + 7) / 8);
  for (int k = 0; k < 6; ++k) {
    int imax = stag_i(k) ? c->d.nr - 1 : c->d.nr, jmax = stag_j(k) ? c->d.nth - 1 : c->d.nth;
    if (which == PIC_FIELDS_TOTAL)
      ++c->launches, k_pack_total<<<gr, dim3(32, 8), 0, c->stream>>>(c->G, c->f[k], tmp + k * plane, k, rows, cols, imax,
                                                                     jmax, c->step * c->G.dt);
    else
      ++c->launches, k_pack<<<gr, dim3(32, 8), 0, c->stream>>>(c->G, c->f[k], tmp + k * plane, 0, rows, cols, imax, jmax, 0);
  }
  int e = to_user(c, tmp, out6, 6 * plane, mem);
  cudaFree(tmp);
  if (e) return e;
  latch_errors(c);
  return status(c);
}

extern "C" int pic_set_fields(pic_ctx *c, const double *in6, int32_t mem) {
  if (!c || !in6) return pic_fail(PIC_EINVAL, "null argument");
  const int rows = c->d.nr + 1, cols = c->d.nth + 1;
  const size_t plane = (size_t)rows * cols;
  double *tmp;
  PIC_CUDA(cudaMalloc((void **)&tmp, 6 * plane * sizeof(double)));
  PIC_CUDA(cudaMemcpyAsync(tmp, in6, 6 * plane * sizeof(double),
                           mem == PIC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  dim3 gr((cols + 31) / 32, (rows + 7) / 8);
  for (int k = 0; k < 6; ++k) {
    int imax = stag_i(k) ? c->d.nr - 1 : c->d.nr, jmax = stag_j(k) ? c->d.nth - 1 : c->d.nth;
    ++c->launches, k_pack<<<gr, dim3(32, 8), 0, c->stream>>>(c->G, c->f[k], tmp + k * plane, 0, rows, cols, imax, jmax, 1);
  }
  fields_fill_ghosts(c);
  PIC_CUDA(cudaStreamSynchronize(c->stream));
  cudaFree(tmp);
  c->have_snap = false;
  return PIC_OK;
}

extern "C" int pic_get_flux(pic_ctx *c, double *out3, int64_t *n, int32_t mem) {
  if (!c || !n) return pic_fail(PIC_EINVAL, "null argument");
  const int g = c->G.g, rows = c->d.nr + 2 * g + 1, cols = c->d.nth + 1;
  const size_t plane = (size_t)rows * cols;
  *n = (int64_t)(3 * plane);
  if (!out3) return PIC_OK;
  double *tmp;
  PIC_CUDA(cudaMalloc((void **)&tmp, 3 * plane * sizeof(double)));
  dim3 gr((cols + 31) / 32, (rows + 7) / 8);
  for (int k = 0; k < 3; ++k)
    ++c->launches, k_pack<<<gr, dim3(32, 8), 0, c->stream>>>(c->G, c->F[k], tmp + k * plane, -g, rows, cols, c->d.nr + g,
                                              k == 1 ? c->d.nth - 1 : c->d.nth, 0);
  int e = to_user(c, tmp, out3, 3 * plane, mem);
  cudaFree(tmp);
  return e;
}

extern "C" int pic_get_charge(pic_ctx *c, int32_t filtered, double *out, int64_t *n, int32_t mem) {
  if (!c || !n) return pic_fail(PIC_EINVAL, "null argument");
  const int g = c->G.g, rows = c->d.nr + 2 * g + 1, cols = c->d.nth + 1;
  const size_t plane = (size_t)rows * cols;
  *n = (int64_t)plane;
  if (!out) return PIC_OK;
  cudaMemsetAsync(c->Q, 0, c->grid_elems * sizeof(double), c->stream);
  cudaMemsetAsync(c->Qa, 0, c->grid_elems * sizeof(double), c->stream);
  if (c->d.precision == PIC_FP32) charge32(c, c->Q, c->Qa);
  else charge64(c, c->Q, c->Qa);
  if (filtered) filter_array(c, c->Q, c->Qt, 0, +1, c->d.n_filt);
  double *tmp;
  PIC_CUDA(cudaMalloc((void **)&tmp, plane * sizeof(double)));
  dim3 gr((cols + 31) / 32, (rows + 7) / 8);
  ++c->launches, k_pack<<<gr, dim3(32, 8), 0, c->stream>>>(c->G, c->Q, tmp, -g, rows, cols, c->d.nr + g, c->d.nth, 0);
  int e = to_user(c, tmp, out, plane, mem);
  cudaFree(tmp);
  if (e) return e;
  latch_errors(c);
  return status(c);
}

extern "C" int pic_grid_coords(pic_ctx *c, int64_t n, const double *r, const double *th, double *x1, double *x2,
                               int32_t mem) {
  if (!c || n < 0) return pic_fail(PIC_EINVAL, "bad argument");
  if (n == 0) return PIC_OK;
  if (!r || !th || !x1 || !x2) return pic_fail(PIC_EINVAL, "null array");
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (mem == PIC_MEM_DEVICE) {
    ++c->launches, k_grid_coords<<<blocks, 256, 0, c->stream>>>(c->G, n, r, th, x1, x2);
    PIC_CUDA(cudaGetLastError());
    PIC_CUDA(cudaStreamSynchronize(c->stream));
    return PIC_OK;
  }
  double *d;
  PIC_CUDA(cudaMalloc((void **)&d, 4 * (size_t)n * sizeof(double)));
  cudaMemcpyAsync(d, r, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(d + n, th, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  ++c->launches, k_grid_coords<<<blocks, 256, 0, c->stream>>>(c->G, n, d, d + n, d + 2 * n, d + 3 * n);
  cudaMemcpyAsync(x1, d + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(x2, d + 3 * n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaError_t err = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  if (err != cudaSuccess) return pic_fail(PIC_ECUDA, cudaGetErrorString(err));
  return PIC_OK;
}

extern "C" int pic_get_particles(pic_ctx *c, int64_t *n, double *x1, double *x2, double *u_r, double *u_th,
                                 double *u_ph, double *qw, int64_t *id, int32_t mem) {
  if (!c || !n) return pic_fail(PIC_EINVAL, "null argument");
  int e = compact(c);
  if (e) return e;
  const int64_t live = c->n_used;
  if (!x1) { *n = live; return status(c); }
  if (*n < live) { *n = live; return pic_fail(PIC_EINVAL, "output buffers too small"); }
  if (!x2 || !u_r || !u_th || !u_ph || !qw) return pic_fail(PIC_EINVAL, "null output array");
  *n = live;
  if (live == 0) return status(c);
  const cudaMemcpyKind kind = mem == PIC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (c->d.precision == PIC_FP64) {
    const size_t b = (size_t)live * 8;
    PIC_CUDA(cudaMemcpyAsync(x1, c->p64.x1, b, kind, c->stream));
    PIC_CUDA(cudaMemcpyAsync(x2, c->p64.x2, b, kind, c->stream));
    PIC_CUDA(cudaMemcpyAsync(u_r, c->p64.ur, b, kind, c->stream));
    PIC_CUDA(cudaMemcpyAsync(u_th, c->p64.ut, b, kind, c->stream));
    PIC_CUDA(cudaMemcpyAsync(u_ph, c->p64.up, b, kind, c->stream));
    PIC_CUDA(cudaMemcpyAsync(qw, c->p64.qw, b, kind, c->stream));
    if (id) PIC_CUDA(cudaMemcpyAsync(id, c->p64.id, b, kind, c->stream));
  } else {
    double *tmp;
    int64_t *tid;
    PIC_CUDA(cudaMalloc((void **)&tmp, 6 * (size_t)live * 8));
    PIC_CUDA(cudaMalloc((void **)&tid, (size_t)live * 8));
    double *t[6];
    for (int k = 0; k < 6; ++k) t[k] = tmp + (size_t)k * live;
    ++c->launches, k_export32<<<(unsigned)((live + 255) / 256), 256, 0, c->stream>>>(c->p32, live, t[0], t[1], t[2], t[3], t[4],
                                                                      t[5], tid);
    double *o[6] = {x1, x2, u_r, u_th, u_ph, qw};
    for (int k = 0; k < 6; ++k) PIC_CUDA(cudaMemcpyAsync(o[k], t[k], (size_t)live * 8, kind, c->stream));
    if (id) PIC_CUDA(cudaMemcpyAsync(id, tid, (size_t)live * 8, kind, c->stream));
    PIC_CUDA(cudaStreamSynchronize(c->stream));
    cudaFree(tmp);
    cudaFree(tid);
  }
  PIC_CUDA(cudaStreamSynchronize(c->stream));
  return status(c);
}

extern "C" int pic_get_moments(pic_ctx *c, pic_moments *out) {
  if (!c || !out) return pic_fail(PIC_EINVAL, "null argument");
  moments(c, false, out);
  PIC_CUDA(cudaGetLastError());
  latch_errors(c);
  return status(c);
}

extern "C" int pic_get_luminosity(pic_ctx *c, double *L, int64_t *n, int32_t mem) {
  if (!c || !n) return pic_fail(PIC_EINVAL, "null argument");
  *n = c->d.nr + 1;
  if (!L) return PIC_OK;
  double *tmp;
  PIC_CUDA(cudaMalloc((void **)&tmp, (size_t)(c->d.nr + 1) * sizeof(double)));
  luminosity(c, c->step * c->G.dt, tmp);
  PIC_CUDA(cudaGetLastError());
  int e = to_user(c, tmp, L, c->d.nr + 1, mem);
  cudaFree(tmp);
  if (e) return e;
  latch_errors(c);
  return status(c);
}

extern "C" int pic_get_live(pic_ctx *c, int64_t *live, double *kinetic_energy) {
  if (!c || !live) return pic_fail(PIC_EINVAL, "null argument");
  cudaMemsetAsync(c->d_acc, 0, ACC_N * sizeof(double), c->stream);
  cudaMemsetAsync(c->d_cnt + CNT_LIVE, 0, sizeof(long long), c->stream);
  if (c->d.precision == PIC_FP32) reduce_particles32(c);
  else reduce_particles64(c);
  long long n = 0;
  double acc[ACC_N];
  PIC_CUDA(cudaMemcpyAsync(&n, c->d_cnt + CNT_LIVE, sizeof n, cudaMemcpyDeviceToHost, c->stream));
  PIC_CUDA(cudaMemcpyAsync(acc, c->d_acc, sizeof acc, cudaMemcpyDeviceToHost, c->stream));
  PIC_CUDA(cudaStreamSynchronize(c->stream));
  *live = n;
  if (kinetic_energy) *kinetic_energy = acc[ACC_KIN];
  latch_errors(c);
  return status(c);
}

extern "C" int pic_gauss_snapshot(pic_ctx *c) {
  if (!c) return pic_fail(PIC_EINVAL, "null context");
  moments(c, true, nullptr);
  PIC_CUDA(cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

extern "C" int pic_set_clock(pic_ctx *c, int64_t step, int64_t next_id) {
  if (!c || step < 0 || next_id < 0) return pic_fail(PIC_EINVAL, "bad clock");
  c->step = step;
  c->next_id = next_id;
  return PIC_OK;
}

extern "C" int pic_profile(pic_ctx *c, int32_t enable) {
  if (!c) return pic_fail(PIC_EINVAL, "null context");
  prof_drain(c);
  c->prof = enable != 0;
  for (int k = 0; k < PROF_N; ++k) { c->prof_ms[k] = 0; c->prof_launch[k] = 0; }
  c->prof_steps = 0;
  return PIC_OK;
}

extern "C" int pic_get_profile(pic_ctx *c, double *ms6, int64_t *steps) {
  if (!c || !ms6) return pic_fail(PIC_EINVAL, "null argument");
  prof_drain(c);
  for (int k = 0; k < PROF_N; ++k) ms6[k] = c->prof_launch[k] ? c->prof_ms[k] / c->prof_launch[k] : 0.0;
  if (steps) *steps = c->prof_steps;
  return PIC_OK;
}

extern "C" int pic_get_axis_ties(pic_ctx *c, int64_t *n, int64_t *steps, int64_t *ids, int32_t *signs) {
  if (!c || !n) return pic_fail(PIC_EINVAL, "null argument");
  long long total = 0;
  PIC_CUDA(cudaMemcpyAsync(&total, c->d_cnt + CNT_TIES, sizeof total, cudaMemcpyDeviceToHost, c->stream));
  PIC_CUDA(cudaStreamSynchronize(c->stream));
  const int64_t logged = std::min<int64_t>(total, TIE_LOG);
  if (!steps) { *n = logged; return PIC_OK; }
  if (*n < logged) { *n = logged; return pic_fail(PIC_EINVAL, "output arrays too small"); }
  if (!ids) return pic_fail(PIC_EINVAL, "null output array");
  *n = logged;
  if (logged == 0) return PIC_OK;
  std::vector<int8_t> sg(logged);
  PIC_CUDA(cudaMemcpy(steps, c->tie_step, logged * sizeof(int64_t), cudaMemcpyDeviceToHost));
  PIC_CUDA(cudaMemcpy(ids, c->tie_id, logged * sizeof(int64_t), cudaMemcpyDeviceToHost));
  PIC_CUDA(cudaMemcpy(sg.data(), c->tie_sign, logged, cudaMemcpyDeviceToHost));
  if (signs)
    for (int64_t k = 0; k < logged; ++k) signs[k] = sg[k];
  return PIC_OK;
}

extern "C" int pic_set_axis_hints(pic_ctx *c, int64_t n, const int64_t *steps, const int64_t *ids,
                                  const int32_t *signs) {
  if (!c || n < 0) return pic_fail(PIC_EINVAL, "bad argument");
  if (n > 0 && (!steps || !ids || !signs)) return pic_fail(PIC_EINVAL, "null hint array");
  PIC_CUDA(cudaStreamSynchronize(c->stream));
  cudaFree(c->hint_step); cudaFree(c->hint_id); cudaFree(c->hint_sign);
  c->hint_step = c->hint_id = nullptr;
  c->hint_sign = nullptr;
  c->nhint = 0;
  if (n == 0) return PIC_OK;
  // sorted by (step, id) for the kernels' binary search
  std::vector<int64_t> ord(n);
  for (int64_t k = 0; k < n; ++k) ord[k] = k;
  std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
    return steps[a] < steps[b] || (steps[a] == steps[b] && ids[a] < ids[b]);
  });
  std::vector<int64_t> hs(n), hi(n);
  std::vector<int8_t> hg(n);
  for (int64_t k = 0; k < n; ++k) {
    hs[k] = steps[ord[k]];
    hi[k] = ids[ord[k]];
    hg[k] = signs[ord[k]] < 0 ? -1 : 1;
  }
  int e;
  if ((e = dalloc(&c->hint_step, n)) || (e = dalloc(&c->hint_id, n)) || (e = dalloc(&c->hint_sign, n))) return e;
  PIC_CUDA(cudaMemcpy(c->hint_step, hs.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice));
  PIC_CUDA(cudaMemcpy(c->hint_id, hi.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice));
  PIC_CUDA(cudaMemcpy(c->hint_sign, hg.data(), n, cudaMemcpyHostToDevice));
  c->nhint = n;
  return PIC_OK;
}

extern "C" int pic_get_launches(pic_ctx *c, int64_t *n) {
  if (!c || !n) return pic_fail(PIC_EINVAL, "null argument");
  *n = c->launches;
  return PIC_OK;
}

// re-bin an FP32 context for another tile shape (sorted at the next step)
int pic_set_tiles(pic_ctx *c, int shape) {
  Tiles &T = c->tiles;
  cudaStreamSynchronize(c->stream);
  cudaFree(T.start);
  cudaFree(T.cursor);
  cudaFree(T.bsum);
  cudaFree(T.ucount);
  cudaFree(T.usum);
  T.start = T.cursor = T.bsum = T.ucount = T.usum = nullptr;
  T.sorted_end = 0;
  T.nunits = 0;
  int e;
  if ((e = alloc_bins(c, shape))) return e;
  c->d.tile_shape = shape;
  c->need_sort = true;
  c->mix_sort = true;
  return PIC_OK;
}

// a new context holding the same fields, particles and clock
int pic_clone_context(pic_ctx *c, pic_ctx **out) {
  pic_desc d = c->d;
  d.capacity = 0;
  int e = pic_init_grid(out, &d, c->stream);
  if (e) return e;
  pic_ctx *k = *out;
  for (int q = 0; q < 6; ++q)
    cudaMemcpyAsync(k->f[q], c->f[q], c->grid_elems * 8, cudaMemcpyDeviceToDevice, c->stream);
  fields_fill_ghosts(k);
  int64_t n = 0;
  if ((e = pic_get_particles(c, &n, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, PIC_MEM_DEVICE)))
    return e;
  if (n > 0) {
    double *buf;
    PIC_CUDA(cudaMalloc((void **)&buf, 6 * (size_t)n * 8));
    double *b[6];
    for (int q = 0; q < 6; ++q) b[q] = buf + (size_t)q * n;
    e = pic_get_particles(c, &n, b[0], b[1], b[2], b[3], b[4], b[5], nullptr, PIC_MEM_DEVICE);
    if (!e) e = pic_load_particles(k, n, b[0], b[1], b[2], b[3], b[4], b[5], PIC_MEM_DEVICE);
    cudaFree(buf);
    if (e) return e;
  }
  // the same fixed-point quantum as the original (its charges may have left)
  cudaMemcpyAsync(k->qexp, c->qexp, sizeof(long long), cudaMemcpyDeviceToDevice, c->stream);
  k->step = c->step;
  k->next_id = c->next_id;
  PIC_CUDA(cudaStreamSynchronize(c->stream));
  return PIC_OK;
}

extern "C" int pic_destroy(pic_ctx *c) {
  if (!c) return PIC_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  free_parts(c);
  cudaFree(c->metric_buf);
  for (int k = 0; k < 6; ++k) { cudaFree(c->f[k]); cudaFree(c->f32[k]); }
  cudaFree(c->r_n32);
  cudaFree(c->th_n32);
  cudaFree(c->d_tile_maps);
  for (int k = 0; k < 3; ++k) { cudaFree(c->F[k]); cudaFree(c->Ft[k]); cudaFree(c->acc[k]); }
  cudaFree(c->Q); cudaFree(c->Qa); cudaFree(c->Qt); cudaFree(c->gsnap); cudaFree(c->sig);
  cudaFree(c->d_err); cudaFree(c->d_cnt); cudaFree(c->d_acc);
  cudaFree(c->tiles.start); cudaFree(c->tiles.cursor); cudaFree(c->tiles.bsum);
  cudaFree(c->tiles.ucount); cudaFree(c->tiles.usum); cudaFree(c->tiles.units);
  cudaFree(c->tie_step); cudaFree(c->tie_id); cudaFree(c->tie_sign);
  cudaFree(c->hint_step); cudaFree(c->hint_id); cudaFree(c->hint_sign);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
  return PIC_OK;
}

// particles64.cu -- the plain FP64 particle path: one thread per particle,
// gather straight from the FP64 field arrays, push and move in Cartesian
// components of the meridional plane, Villasenor-Buneman deposit with FP64
// global atomics.  Also: stable removal of deleted particles and the particle
// reductions used by the diagnostics.
#include "pic_internal.h"

namespace pic {

namespace {

__device__ inline int cell_j(const Grid &G, double x2) {
  int j = (int)floor(x2);
  return j > G.nth - 1 ? G.nth - 1 : (j < 0 ? 0 : j);
}

// bilinear interpolation in grid coordinates from a component's staggered
// lattice (reading of the gather; the axis and conductor ghosts are stored);
// x1 is the slab's local coordinate (global - i0, an exact difference)
__device__ inline double interp64(const Grid &G, const double *__restrict__ a, double x1, double x2, int si, int sj) {
  const double p1 = x1 - 0.5 * si, p2 = x2 - 0.5 * sj;
  const double fi = floor(p1), fj = floor(p2);
  const double w1 = p1 - fi, w2 = p2 - fj;
  const size_t o = gidx(G, (int)fi, (int)fj);
  return (1 - w1) * (1 - w2) * a[o] + w1 * (1 - w2) * a[o + G.LD] + (1 - w1) * w2 * a[o + 1] +
         w1 * w2 * a[o + G.LD + 1];
}

// charge crossing the four dual faces around cell (ic, jc) for a straight path
// p -> q inside that cell (Villasenor-Buneman, Eq. Jcons)
__device__ inline void vb_seg64(const Grid &G, double *Fr, double *Ft, double qw, int ic, int jc, double p1, double p2,
                                double q1, double q2) {
  const double d1 = q1 - p1, d2 = q2 - p2;
  const double m1 = 0.5 * (p1 + q1) - ic, m2 = 0.5 * (p2 + q2) - jc;
  const size_t o = gidx(G, ic, jc);
  atomicAdd(Fr + o, qw * d1 * (1.0 - m2));
  atomicAdd(Fr + o + 1, qw * d1 * m2);
  atomicAdd(Ft + o, qw * d2 * (1.0 - m1));
  atomicAdd(Ft + o + G.LD, qw * d2 * m1);
}

__device__ inline double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

// the path a -> b split where it crosses grid lines (at most one per direction)
__device__ inline void vb_path64(const Grid &G, double *Fr, double *Ft, double qw, double a1, double a2, double b1,
                                 double b2, int ia, int ib) {
  const int ja = cell_j(G, a2), jb = cell_j(G, b2);
  const int X = ia > ib ? ia : ib, Y = ja > jb ? ja : jb;
  double sx = 2.0, sy = 2.0;
  if (ib != ia) sx = (X - a1) / (b1 - a1);
  if (jb != ja) sy = (Y - a2) / (b2 - a2);
  double P1 = a1, P2 = a2;
  int ic = ia, jc = ja;
#pragma unroll
  for (int ev = 0; ev < 2; ++ev) {
    const bool xf = sx <= sy;
    const double sn = xf ? sx : sy;
    if (sn > 1.0) break;
    double Q1, Q2;
    if (xf) { Q1 = X; Q2 = clampd(a2 + sn * (b2 - a2), jc, jc + 1); }
    else { Q2 = Y; Q1 = clampd(a1 + sn * (b1 - a1), ic, ic + 1); }
    vb_seg64(G, Fr, Ft, qw, ic, jc, P1, P2, Q1, Q2);
    P1 = Q1; P2 = Q2;
    if (xf) { ic = ib; sx = 2.0; } else { jc = jb; sy = 2.0; }
  }
  vb_seg64(G, Fr, Ft, qw, ic, jc, P1, P2, b1, b2);
}

struct Fields64 { const double *f[6]; };
struct Flux64 { double *Fr, *Ft, *Fp; };

__global__ void __launch_bounds__(256) k_particles64(Grid G, Parts64 P, int64_t n, double t, Fields64 F, Flux64 D,
                                                     int *err, long long *cnt, AxisTies ties) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double qw = P.qw[k];
  if (qw == 0.0) return;  // free slot
  const double x1 = P.x1[k], x2 = P.x2[k];
  const double r = map_r(G, x1), th = map_th(G, x2);
  double st, ct;
  sincos(th, &st, &ct);
  const double ur = P.ur[k], ut = P.ut[k], up = P.up[k];
  // local spherical basis at phi = 0 -> Cartesian (x = R, y = phi, z)
  double u[3] = {ur * st + ut * ct, up, ur * ct - ut * st};
  // physical tests in global coordinates, array indices in the slab's rows
  const double xl = x1 - (double)G.i0;
  if (x1 < G.nr_glob) {  // inside the outer conductor particles fly ballistically
    double Es[3], Bs[3];
    const Vac<double> V{G.vacuum, G.b0, G.r_min, omega_at(G.omega, G.t_spin, t)};
    vacuum_field<double>(V, r, st, ct, x1 < 0.0, Es, Bs);
    if (x1 >= 0.0) {  // no plasma field inside the inner conductor
      Es[0] += interp64(G, F.f[ER], xl, x2, 1, 0);
      Es[1] += interp64(G, F.f[ETH], xl, x2, 0, 1);
      Es[2] += interp64(G, F.f[EPH], xl, x2, 0, 0);
      Bs[0] += interp64(G, F.f[BR], xl, x2, 0, 1);
      Bs[1] += interp64(G, F.f[BTH], xl, x2, 1, 0);
      Bs[2] += interp64(G, F.f[BPH], xl, x2, 1, 1);
    }
    const double E[3] = {Es[0] * st + Es[1] * ct, Es[2], Es[0] * ct - Es[1] * st};
    const double B[3] = {Bs[0] * st + Bs[1] * ct, Bs[2], Bs[0] * ct - Bs[1] * st};
    push<double>(G.pusher, (qw > 0.0 ? 1.0 : -1.0) * G.qm * G.dt, E, B, u);
  }
  // straight 3-D move from (r st, 0, r ct), then back to phi = 0 (Sec. 3.3)
  const double ig = 1.0 / sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  const double X = r * st + u[0] * ig * G.dt, Y = u[1] * ig * G.dt, Z = r * ct + u[2] * ig * G.dt;
  const double R = hypot(X, Y), rn = hypot(R, Z), thn = atan2(R, Z);
  double phi = atan2(Y, X);
  if (X < 0.0 && u[1] * u[1] <= (AXIS_TIE * AXIS_TIE) * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]))
    phi = axis_tie(ties, P.id[k], phi);  // rare: see AxisTies
  const double cp = R > 0.0 ? X / R : 1.0, sp = R > 0.0 ? Y / R : 0.0;
  const double ux = cp * u[0] + sp * u[1], uy = -sp * u[0] + cp * u[1], uz = u[2];
  const double stn = rn > 0.0 ? R / rn : 0.0, ctn = rn > 0.0 ? Z / rn : 1.0;
  double nx1 = map_r_inv(G, rn), nx2 = clampd(map_th_inv(G, thn), 0.0, (double)G.nth);
  const double nur = ux * stn + uz * ctn, nut = ux * ctn - uz * stn;
  if (!(isfinite(nx1) && isfinite(nx2) && isfinite(nur) && isfinite(nut) && isfinite(uy))) {
    set_err(err, ERR_NAN);
    P.qw[k] = 0.0;
    return;
  }
  const int ia = (int)floor(x1);
  const double lo = -(double)G.g, hi = (double)(G.nr_glob + G.g);
  if (!(nx1 >= lo && nx1 < hi) || abs((int)floor(nx1) - ia) > 1 || abs(cell_j(G, nx2) - cell_j(G, x2)) > 1) {
    set_err(err, ERR_COURANT);
  } else {
    const double nxl = nx1 - (double)G.i0;
    const int ib = (int)floor(nx1);
    vb_path64(G, D.Fr, D.Ft, qw, xl, x2, nxl, nx2, ia - G.i0, ib - G.i0);
    // azimuthal flux: charge crossing the meridional half-plane, area weights
    // at the midpoint of the grid-coordinate path (reading of the paper)
    const double m1 = 0.5 * (xl + nxl), m2 = 0.5 * (x2 + nx2);
    const double fi = floor(m1), fj = floor(m2), w1 = m1 - fi, w2 = m2 - fj;
    const double v = qw * phi * (0.5 / PI_D);
    const size_t o = gidx(G, (int)fi, (int)fj);
    atomicAdd(D.Fp + o, v * (1 - w1) * (1 - w2));
    atomicAdd(D.Fp + o + G.LD, v * w1 * (1 - w2));
    atomicAdd(D.Fp + o + 1, v * (1 - w1) * w2);
    atomicAdd(D.Fp + o + G.LD + 1, v * w1 * w2);
  }
  // removal once the filtered shape lies inside a conductor (Sec. 3.4.2)
  const int ci = (int)floor(nx1);
  if (ci < -(G.n_filt + 1) || ci >= G.nr_glob + G.n_filt + 1) {
    P.qw[k] = 0.0;
    add_ll(cnt + CNT_DELETED, 1LL);
    return;
  }
  P.x1[k] = nx1;
  P.x2[k] = nx2;
  P.ur[k] = nur;
  P.ut[k] = nut;
  P.up[k] = uy;
}

// ---- stable removal of free slots (block counts, one-block scan, scatter) ----
constexpr int CB = 256;

__global__ void k_count_live(const double *__restrict__ qw, int64_t n, long long *bc) {
  const int64_t k = blockIdx.x * (int64_t)CB + threadIdx.x;
  int live = (k < n && qw[k] != 0.0) ? 1 : 0;
  int s = __syncthreads_count(live);
  if (threadIdx.x == 0) bc[blockIdx.x] = s;
}

__global__ void k_scan_blocks(long long *bc, int64_t nb, long long *total) {
  // exclusive scan of nb block counts by one block of 1024 threads
  __shared__ long long part[1024];
  const int t = threadIdx.x;
  const int64_t per = (nb + 1023) / 1024, b0 = t * per, b1 = min(nb, b0 + per);
  long long s = 0;
  for (int64_t b = b0; b < b1; ++b) s += bc[b];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    long long v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  long long run = part[t] - s;
  for (int64_t b = b0; b < b1; ++b) {
    long long c = bc[b];
    bc[b] = run;
    run += c;
  }
  if (t == 1023) *total = part[1023];
}

__global__ void k_scatter_live(Parts64 S, Parts64 D, int64_t n, const long long *__restrict__ boff) {
  __shared__ int wsum[CB / 32];
  const int64_t k = blockIdx.x * (int64_t)CB + threadIdx.x;
  const int live = (k < n && S.qw[k] != 0.0) ? 1 : 0;
  const unsigned m = __ballot_sync(0xffffffffu, live);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int before = __popc(m & ((1u << lane) - 1u));
  if (lane == 0) wsum[w] = __popc(m);
  __syncthreads();
  int base = 0;
  for (int q = 0; q < w; ++q) base += wsum[q];
  if (live) {
    const int64_t d = boff[blockIdx.x] + base + before;
    D.x1[d] = S.x1[k]; D.x2[d] = S.x2[k];
    D.ur[d] = S.ur[k]; D.ut[d] = S.ut[k]; D.up[d] = S.up[k];
    D.qw[d] = S.qw[k]; D.id[d] = S.id[k];
  }
}

__global__ void k_charge64(Grid G, const double *__restrict__ x1, const double *__restrict__ x2,
                           const double *__restrict__ qw, int64_t n, double *Q, double *Qa) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double q = qw[k];
  if (q == 0.0) return;
  const double a = x1[k] - (double)G.i0, b = x2[k], fi = floor(a), fj = floor(b), w1 = a - fi, w2 = b - fj;
  const size_t o = gidx(G, (int)fi, (int)fj);
  const double c00 = (1 - w1) * (1 - w2), c10 = w1 * (1 - w2), c01 = (1 - w1) * w2, c11 = w1 * w2;
  atomicAdd(Q + o, q * c00); atomicAdd(Q + o + G.LD, q * c10);
  atomicAdd(Q + o + 1, q * c01); atomicAdd(Q + o + G.LD + 1, q * c11);
  const double aq = fabs(q);
  atomicAdd(Qa + o, aq * c00); atomicAdd(Qa + o + G.LD, aq * c10);
  atomicAdd(Qa + o + 1, aq * c01); atomicAdd(Qa + o + G.LD + 1, aq * c11);
}

__global__ void k_reduce64(Parts64 P, int64_t n, double qm, double *acc, long long *live) {
  double kin = 0.0, ch = 0.0;
  long long l = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    if (P.qw[k] == 0.0) continue;
    const double q = P.qw[k], u2 = P.ur[k] * P.ur[k] + P.ut[k] * P.ut[k] + P.up[k] * P.up[k];
    kin += fabs(q) / qm * (sqrt(1.0 + u2) - 1.0);
    ch += q;
    l += 1;
  }
  block_sum3(kin, ch, l, acc + ACC_KIN, acc + ACC_CHARGE, live);
}

}  // namespace

void particles64(pic_ctx *c, double t) {
  if (c->n_used == 0) return;
  Fields64 F;
  for (int k = 0; k < 6; ++k) F.f[k] = c->f[k];
  Flux64 D{c->F[0], c->F[1], c->F[2]};
  const int64_t blocks = (c->n_used + 255) / 256;
  ++c->launches, k_particles64<<<(unsigned)blocks, 256, 0, c->stream>>>(c->G, c->p64, c->n_used, t, F, D, c->d_err, c->d_cnt,
                                                                          axis_ties(c));
}

int64_t compact64(pic_ctx *c) {
  const int64_t n = c->n_used;
  if (n == 0) return 0;
  const int64_t nb = (n + CB - 1) / CB;
  long long *bc = (long long *)c->scratch;
  ++c->launches, k_count_live<<<(unsigned)nb, CB, 0, c->stream>>>(c->p64.qw, n, bc);
  ++c->launches, k_scan_blocks<<<1, 1024, 0, c->stream>>>(bc, nb, c->d_cnt + CNT_SORTED);
  ++c->launches, k_scatter_live<<<(unsigned)nb, CB, 0, c->stream>>>(c->p64, c->q64, n, bc);
  cudaMemcpyAsync(c->h_pinned, c->d_cnt + CNT_SORTED, sizeof(long long), cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  const int64_t live = *c->h_pinned;
  Parts64 t = c->p64;
  c->p64 = c->q64;
  c->q64 = t;
  c->n_used = live;
  return live;
}

void charge64(pic_ctx *c, double *Q, double *Qa) {
  if (c->n_used == 0) return;
  ++c->launches, k_charge64<<<(unsigned)((c->n_used + 255) / 256), 256, 0, c->stream>>>(c->G, c->p64.x1, c->p64.x2, c->p64.qw,
                                                                        c->n_used, Q, Qa);
}

void reduce_particles64(pic_ctx *c) {
  if (c->n_used == 0) return;
  // a fixed grid (4 blocks per SM) keeps the same-address atomics few
  ++c->launches, k_reduce64<<<4 * 152, 256, 0, c->stream>>>(c->p64, c->n_used, c->G.qm, c->d_acc,
                                                                        c->d_cnt + CNT_LIVE);
}

}  // namespace pic

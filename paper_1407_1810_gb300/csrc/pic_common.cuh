// pic_common.cuh -- device-side definitions shared by the library's kernels.
//
// Layout in HBM: every grid quantity (6 field components, 3 charge fluxes,
// node charge, FP32 field copies, fixed-point flux accumulators) is one 2-D
// row-major array over the same padded index space:
//   rows i in [-PI, nr + PI), columns j in [-PJ, nth + PJ), stride LD,
//   element (i, j) at (i + PI) * LD + (j + PJ).
// Index (i, j) of a component names its staggered point of Eq. (offseteq).
// Rows outside [0, nr] are the conductor interiors: field values there are 0,
// flux rows -g..nr+g (g = n_filt + 2) receive the deposit of particles inside
// the conductors (Sec. 3.4.2).  Columns -1 and nth of the half-integer-j
// components hold their axisymmetric continuation across the polar axis
// (B_r even, E_th and B_ph odd), so a gather never branches on the axis.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pic {

constexpr int PAD = 40;  // padding rows/columns on each side: covers every tile window (tile side + halo <= PAD)

enum Comp { ER = 0, ETH = 1, EPH = 2, BR = 3, BTH = 4, BPH = 5 };
// staggering of Eq. (offseteq): 1 = half-integer position
__host__ __device__ constexpr int stag_i(int c) { return (c == ER || c == BTH || c == BPH) ? 1 : 0; }
__host__ __device__ constexpr int stag_j(int c) { return (c == ETH || c == BR || c == BPH) ? 1 : 0; }

enum ErrBits { ERR_COURANT = 1, ERR_CAPACITY = 2, ERR_NAN = 4, ERR_RANGE = 8, ERR_TIMEOUT = 16 };

// Row/column metric tables (FP64), each indexed by i + PI or j + PJ.
struct Metric {
  const double *r_n, *r_h;          // f_r(i), f_r(i + 1/2)
  const double *inv_r_n;            // 1 / r_i
  const double *inv_dr2_n;          // 2 / (r_{i+1}^2 - r_i^2)
  const double *dr_n;               // r_{i+1} - r_i
  const double *inv_r_h;            // 1 / rb_i
  const double *inv_area_h;         // 1 / (2 pi rb_i^2)
  const double *inv_dr2_h;          // 2 / (rb_i^2 - rb_{i-1}^2)
  const double *dr_h;               // rb_i - rb_{i-1}
  const double *keep_n, *keep_h;    // 1 - sigma*(i), 1 - sigma*(i + 1/2)  (Eq. EBcond)
  const double *vol_r_n, *vol_r_h;  // radial factors of the cell volumes (energy)
  const double *sin_t;              // sin th_j
  const double *cos_t;              // cos th_j
  const double *inv_dcos_t;         // 1 / (cos th_j - cos th_{j+1})
  const double *inv_dth_t;          // 1 / (th_{j+1} - th_j)
  const double *sin_tb;             // sin tb_j, with sin tb_{-1} = sin tb_{nth} = 0
  const double *cos_tb;             // cos tb_j (j < nth)
  const double *inv_sin_tb;         // 1 / sin tb_j
  const double *inv_dcos_tb;        // 1 / (cos tb_{j-1} - cos tb_j), caps at j = 0, nth
  const double *inv_dtb;            // 1 / (tb_j - tb_{j-1})
  const double *vol_t_n, *vol_t_h;  // meridional factors of the cell volumes
  // the Yee update's factors folded into per-row and per-column coefficients
  // (h = dt / 2 for the B half steps, dt for E), so each node costs a few FMAs
  const double *bR;                 // h / r_i                                  (B_r)
  const double *bT0, *bT1;          // h 2 r_i / (r_{i+1}^2 - r_i^2), same with r_{i+1}  (B_th, B_ph)
  const double *bP;                 // h 2 (r_{i+1} - r_i) / (r_{i+1}^2 - r_i^2)  (B_ph)
  const double *eR;                 // dt / rb_i                                (E_r)
  const double *eT0, *eT1;          // dt 2 rb_{i-1} / (rb_i^2 - rb_{i-1}^2), same with rb_i  (E_th, E_ph)
  const double *eP;                 // dt 2 (rb_i - rb_{i-1}) / (rb_i^2 - rb_{i-1}^2)  (E_ph)
  const double *cB1, *cB2;          // sin th_j / dcos_j, sin th_{j+1} / dcos_j  (B_r)
  const double *cE1, *cE2;          // sin tb_j / dcos_tb_j, sin tb_{j-1} / dcos_tb_j  (E_r)
  const double *cF;                 // 1 / (2 pi sin tb_j)                      (E_th flux)
};

struct Grid {
  int nr, nth, g, n_filt;
  // radial slab of a larger grid (Sec. 2: the grid split among processes):
  // local row i is global row i + i0 of a grid of nr_glob rows; particles keep
  // global coordinates, arrays and the row loops use local rows.  An open
  // side is an interface to a neighbouring slab, not a conductor.  A whole
  // grid has i0 = 0, nr_glob = nr and both sides closed.
  int i0, nr_glob, open_lo, open_hi;
  int PI, PJ, LD;
  int r_map, th_map;
  double r_min, dxi;  // log: ln(r_max/r_min)/nr ; linear: (r_max - r_min)/nr
  double dt, qm;
  int vacuum, pusher;
  double b0, omega, t_spin;
  int absorb_cells;
  Metric m;
};

__host__ __device__ inline size_t gidx(const Grid &G, int i, int j) {
  return (size_t)(i + G.PI) * (size_t)G.LD + (size_t)(j + G.PJ);
}

constexpr double PI_D = 3.14159265358979323846;

// ---- stretching functions, Sec. 3.2 -----------------------------------------
__device__ inline double map_r(const Grid &G, double x1) {
  return G.r_map == 1 ? G.r_min * exp(x1 * G.dxi) : G.r_min + x1 * G.dxi;
}
__device__ inline double map_r_inv(const Grid &G, double r) {
  return G.r_map == 1 ? log(r / G.r_min) / G.dxi : (r - G.r_min) / G.dxi;
}
__device__ inline double map_th(const Grid &G, double x2) {
  return G.th_map == 1 ? acos(1.0 - 2.0 * x2 / G.nth) : PI_D * x2 / G.nth;
}
__device__ inline double map_th_inv(const Grid &G, double th) {
  return G.th_map == 1 ? 0.5 * G.nth * (1.0 - cos(th)) : th * G.nth / PI_D;
}

// reciprocal and reciprocal square root: hardware approximations (within 2
// ulp) in FP32, exact division in FP64
__device__ inline float rcp_(float x) { return __fdividef(1.0f, x); }
__device__ inline double rcp_(double x) { return 1.0 / x; }
__device__ inline float rsqrt_(float x) { return rsqrtf(x); }
__device__ inline double rsqrt_(double x) { return 1.0 / sqrt(x); }

// ---- analytic "initial" fields: Sec. 5.2 (monopole, rotator inside/outside),
//      Sec. 4.3 (dipole + corotation), uniform B_z.  Spherical components.
//      W = Omega(t)/c after the linear spin-up. -----------------------------------
template <typename T>
struct Vac {
  int kind;
  T b0, r0, W;
};

__host__ __device__ inline double omega_at(double omega, double t_spin, double t) {
  return (t_spin > 0.0 && t < t_spin) ? omega * (t / t_spin) : omega;
}

template <typename T>
__device__ inline void vacuum_field(const Vac<T> &V, T r, T st, T ct, bool inside, T E[3], T B[3]) {
  E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = T(0);
  if (V.kind == 0) return;
  const T b0 = V.b0, r0 = V.r0, W = V.W;
  const T ir = rcp_(r), q = r0 * ir;
  switch (V.kind) {
    case 1:  // monopole
      B[0] = b0 * q * q;
      break;
    case 2:  // rotating monopole
      B[0] = b0 * q * q;
      if (!inside) {
        T a = b0 * (q * q) * (q * r0) * W;  // b0 r0^4 / r^3 * Omega
        E[0] = T(-2) * a * ct;
        E[1] = -a * st;
      } else {
        E[1] = -b0 * r0 * q * W * st;  // b0 r0^2 / r * Omega
      }
      break;
    case 3:  // uniform B along +z
      B[0] = b0 * ct;
      B[1] = -b0 * st;
      break;
    case 4: {  // dipole + corotation
      T mu = b0 * r0 * r0 * r0, ir3 = ir * ir * ir;
      B[0] = T(2) * mu * ct * ir3;
      B[1] = mu * st * ir3;
      E[0] = mu * W * st * st * ir * ir;
      E[1] = -mu * W * T(2) * st * ct * ir * ir;
      break;
    }
    case 5: {  // aligned dipole rotator: corotation inside, l = 2 vacuum field outside
      T mu = b0 * r0 * r0 * r0, ir2 = ir * ir;
      B[0] = T(2) * mu * ct * ir2 * ir;
      B[1] = mu * st * ir2 * ir;
      if (inside) {
        E[0] = mu * W * st * st * ir2;
        E[1] = -mu * W * T(2) * st * ct * ir2;
      } else {
        T a = mu * W * (q * q) * ir2;  // Omega mu r0^2 / r^4
        E[0] = -a * (T(3) * ct * ct - T(1));
        E[1] = -a * T(2) * st * ct;
      }
      break;
    }
    default:
      break;
  }
}

// ---- pushers, Sec. 2 (Boris 1970; Vay 2008).  Any right-handed orthonormal
//      basis; qmdt = (q/m) dt.  u = gamma v updated in place. -------------------
template <typename T>
__device__ inline void push_boris(T qmdt, const T E[3], const T B[3], T u[3]) {
  const T h = T(0.5) * qmdt;
  T um0 = u[0] + h * E[0], um1 = u[1] + h * E[1], um2 = u[2] + h * E[2];
  T ig = rsqrt_(T(1) + um0 * um0 + um1 * um1 + um2 * um2);
  T t0 = h * B[0] * ig, t1 = h * B[1] * ig, t2 = h * B[2] * ig;
  T f = T(2) * rcp_(T(1) + t0 * t0 + t1 * t1 + t2 * t2);
  T up0 = um0 + (um1 * t2 - um2 * t1), up1 = um1 + (um2 * t0 - um0 * t2), up2 = um2 + (um0 * t1 - um1 * t0);
  T s0 = f * t0, s1 = f * t1, s2 = f * t2;
  u[0] = um0 + (up1 * s2 - up2 * s1) + h * E[0];
  u[1] = um1 + (up2 * s0 - up0 * s2) + h * E[1];
  u[2] = um2 + (up0 * s1 - up1 * s0) + h * E[2];
}

template <typename T>
__device__ inline void push_vay(T qmdt, const T E[3], const T B[3], T u[3]) {
  const T h = T(0.5) * qmdt;
  T ig0 = rsqrt_(T(1) + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  T tau0 = h * B[0], tau1 = h * B[1], tau2 = h * B[2];
  T v0 = u[0] * ig0, v1 = u[1] * ig0, v2 = u[2] * ig0;
  // u' = u + (q dt/m) E + v x tau
  T a0 = u[0] + qmdt * E[0] + (v1 * tau2 - v2 * tau1);
  T a1 = u[1] + qmdt * E[1] + (v2 * tau0 - v0 * tau2);
  T a2 = u[2] + qmdt * E[2] + (v0 * tau1 - v1 * tau0);
  T tau2s = tau0 * tau0 + tau1 * tau1 + tau2 * tau2;
  T ustar = a0 * tau0 + a1 * tau1 + a2 * tau2;
  T sigma = T(1) + a0 * a0 + a1 * a1 + a2 * a2 - tau2s;
  T g2 = T(0.5) * (sigma + sqrt(sigma * sigma + T(4) * (tau2s + ustar * ustar)));
  T ig = rsqrt_(g2);
  T t0 = tau0 * ig, t1 = tau1 * ig, t2 = tau2 * ig;
  T s = rcp_(T(1) + t0 * t0 + t1 * t1 + t2 * t2);
  T at = a0 * t0 + a1 * t1 + a2 * t2;
  u[0] = s * (a0 + at * t0 + (a1 * t2 - a2 * t1));
  u[1] = s * (a1 + at * t1 + (a2 * t0 - a0 * t2));
  u[2] = s * (a2 + at * t2 + (a0 * t1 - a1 * t0));
}

template <typename T>
__device__ inline void push(int pusher, T qmdt, const T E[3], const T B[3], T u[3]) {
  if (pusher == 1) push_boris(qmdt, E, B, u);
  else push_vay(qmdt, E, B, u);
}

// ---- ties of the azimuth branch at the polar axis (Sec. 3.3, reading of the
//      azimuthal flux) -------------------------------------------------------
// A move that carries a particle across the polar axis (Px < 0, the
// displaced point's coordinate along the old cylindrical radius) sweeps an
// azimuth atan2(Dp, Px) whose sign is that of u_ph, and the two signs differ
// by up to 2 pi: the azimuthal flux jumps by up to the particle's whole
// charge as u_ph passes through zero.  When |u_ph| <= AXIS_TIE |u| the sign is
// set by the rounding of a nearly vanishing u_ph and either branch is a valid
// result.  Such ties are counted and logged as (step, id, sign).  A table of
// hints, taken from the log of another run, fixes the branch of the ties it
// lists, so that a replay follows the run it is compared with.
constexpr double AXIS_TIE = 1.0 / 8192;
struct AxisTies {
  const int64_t *hstep = nullptr, *hid = nullptr;  // hints, sorted by (step, id)
  const int8_t *hsign = nullptr;
  int64_t nh = 0;
  int64_t *lstep = nullptr, *lid = nullptr;        // the log of this run
  int8_t *lsign = nullptr;
  int64_t lcap = 0;
  long long *count = nullptr;                      // ties met (the log keeps the first lcap)
  int64_t step = 0;                                // the step being taken
};

// the branch of a tie: the hinted sign if (step, id) is in the table, else
// phi's own; logged; returns +-|phi|
template <typename T>
__device__ inline T axis_tie(const AxisTies &X, int64_t id, T phi) {
  int sg = phi < T(0) ? -1 : 1;
  int64_t lo = 0, hi = X.nh;
  while (lo < hi) {  // first entry not below (step, id)
    const int64_t mid = (lo + hi) >> 1;
    const bool below = X.hstep[mid] < X.step || (X.hstep[mid] == X.step && X.hid[mid] < id);
    if (below) lo = mid + 1;
    else hi = mid;
  }
  if (lo < X.nh && X.hstep[lo] == X.step && X.hid[lo] == id) sg = X.hsign[lo] < 0 ? -1 : 1;
  const long long n = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(X.count), 1ull);
  if (n < X.lcap) { X.lstep[n] = X.step; X.lid[n] = id; X.lsign[n] = (int8_t)sg; }
  return sg > 0 ? fabs(phi) : -fabs(phi);
}

__device__ inline void set_err(int *err, int bits) { atomicOr(err, bits); }
// block-wide sums of (double, double, int) with one atomic per block:
// warp shuffles, then the warp leaders through shared memory
__device__ inline void block_sum3(double a, double b, long long n, double *pa, double *pb, long long *pn) {
  __shared__ double sa[32], sb[32];
  __shared__ long long sn[32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    n += __shfl_xor_sync(0xffffffffu, n, o);
  }
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) { sa[w] = a; sb[w] = b; sn[w] = n; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    long long tn = 0;
    for (int k = 0; k < nw; ++k) { ta += sa[k]; tb += sb[k]; tn += sn[k]; }
    if (pa) atomicAdd(pa, ta);
    if (pb) atomicAdd(pb, tb);
    if (pn) atomicAdd(reinterpret_cast<unsigned long long *>(pn), static_cast<unsigned long long>(tn));
  }
}
// signed 64-bit add through the unsigned overload (two's complement)
__device__ inline void add_ll(long long *p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
}

}  // namespace pic

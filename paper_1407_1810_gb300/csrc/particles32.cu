// particles32.cu -- the FP32 cell+offset particle path (the hot path):
//
//  * particles are kept binned by tiles of TI x TJ cells (counting sort by tile,
//    every sort_interval steps; deleted particles are dropped by the sort);
//  * one CTA per tile stages a window of the FP32 field copies (tile + halo H
//    + the stencil) in shared memory, gathers, pushes and moves every particle
//    of its bin, and deposits the Villasenor-Buneman fluxes into shared-memory
//    int64 fixed-point accumulators (exact and order independent), flushed
//    with one global atomic per nonzero window node;
//  * a particle that drifted out of its tile's window since the last sort, or
//    was injected after it, takes the same code with global-memory accessors.
//
// Position = integer cell + FP32 offset in [0, 1).  The move runs in the
// particle's local frame: the radial increment comes from log1p of the
// relative displacement, the meridional one from the exact rotation angle of
// the displaced point, so an offset keeps ~1e-7 cell accuracy anywhere on the
// grid instead of the ~1e-4 cell an absolute FP32 r or theta would give.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda.h>  // CUtensorMap (the encoder is reached through the runtime's driver entry point)

#include "pic_internal.h"

namespace pic {

namespace {

// halo cells around a tile served from shared memory.  A particle that
// drifts beyond it between sorts takes the global-memory path, and one such
// lane makes its whole warp run that path: with 4 cells (0.003 % of
// particle-steps at 20 steps per sort, against 0.14 % with 2) the window of
// 27 x 27 nodes still leaves room for 4 CTAs per SM.
constexpr int H = 4;
// the last tile of a row or column reaches up to its side + H + 1 nodes past
// the grid's ghost band: the padding of the grid arrays must hold it for the
// longest tile side (32 cells), so the window stays inside the allocation
static_assert(32 + H + 1 <= PAD, "grid padding must cover every tile window");
// window nodes of a TI x TJ tile: the tile, the halo and the stencil reach
template <int TI, int TJ>
struct Win {
  static constexpr int WI = TI + 2 * H + 3, WJ = TJ + 2 * H + 3, WN = WI * WJ;
};
constexpr int NT = 256;                                  // threads per tile CTA
// Shared-memory accumulation splits each term v (|v| <= 2^36 quanta) into
// v = h 2^SPLIT + l with |h| <= 2^18, |l| <= 2^17 and sums h and l with
// native 32-bit shared atomics: both sums stay exact below 2^31 / 2^18 = 8192
// terms per node per tile per step (about 2000 particles per cell); sums
// approaching that limit are reported as ERR_CAPACITY.
constexpr int SPLIT = 18;

struct Args32 {
  int nr, nth, n_filt, PI, PJ, LD;
  int r_log, th_ea, vacuum, pusher;
  float dxi, inv_dxi, dt, qm, inv_nth, nth_f;
  // constants carried as FP32 hi + lo pairs: a constant rounded once to FP32
  // would bias every particle's step the same way (a systematic error that
  // grows linearly with the step count)
  float dt_lo, inv_dxi_lo, k2_hi, k2_lo;  // k2 = nth / pi (linear theta map)
  float b0_lo, qmdt;     // qmdt = (q/m) dt rounded once
  float pi_nth;          // pi / nth (linear theta map: angle per column)
  const long long *qexp;    // fixed-point exponent e: one flux unit is 2^(e - KFIX)
  const int64_t *ids;       // particle ids (read only for an axis-crossing tie)
  AxisTies ties;
  const float *r_n;         // f_r(i) per padded row (FP32)
  const float2 *th_n;       // (sin, cos) of the node angle per padded column (FP32, linear theta map)
  const float *f[6];        // FP32 field copies (padded)
  long long *acc[3];        // global fixed-point flux accumulators (padded)
  int *err;
  long long *cnt;
  // tiles
  int row0, ntj, ntiles, ti, tj, tc;
  int mix;                  // sort: 1 = by cell, bins stored transposed; 0 = by tile, order kept
  const int64_t *start;
  const long long *units;   // work units: tile << 32 | index of the unit within its tile
  int64_t nunits, unit;     // units of the binned particles; particles per unit
  int64_t sorted_end, n_used;
  // vacuum
  float b0, r_min, omega_t;
};

__device__ inline size_t pidx(const Args32 &A, int i, int j) {
  return (size_t)(i + A.PI) * (size_t)A.LD + (size_t)(j + A.PJ);
}

template <int WJ, int WN>
struct SmemAcc {  // window accessors (shared memory)
  const float *f;           // 6 * WN
  int *hi;                  // 3 * WN : sums of the high parts
  int *lo;                  // 3 * WN : sums of the low parts
  const float *rn;          // f_r(i) of the window's rows
  const float2 *tn;         // (sin, cos) of the node angles of the window's columns
  int wi0, wj0;
  float fs;                 // flux units per unit charge, 2^(KFIX - e)
  __device__ float fld(int c, int i, int j) const { return f[c * WN + (i - wi0) * WJ + (j - wj0)]; }
  __device__ float rad(int i) const { return rn[i - wi0]; }
  __device__ float2 ang(int j) const { return tn[j - wj0]; }
  // unconditional: a test for zero terms would branch around every atomic,
  // which costs more than adding the rare zero
  __device__ void add(int k, int i, int j, int h, int l) const {
    const int e = k * WN + (i - wi0) * WJ + (j - wj0);
    atomicAdd(&hi[e], h);
    atomicAdd(&lo[e], l);
  }
};

struct GlobAcc {  // global-memory accessors (particles outside the window)
  const Args32 *A;
  float fs;
  __device__ float fld(int c, int i, int j) const { return A->f[c][pidx(*A, i, j)]; }
  __device__ float rad(int i) const { return A->r_n[i + A->PI]; }
  __device__ float2 ang(int j) const { return A->th_n[j + A->PJ]; }
  __device__ void add(int k, int i, int j, int h, int l) const {
    const long long v = ((long long)h << SPLIT) + (long long)l;
    if (v) atomicAdd(reinterpret_cast<unsigned long long *>(A->acc[k] + pidx(*A, i, j)), (unsigned long long)v);
  }
};

// Fixed-point split of a flux term cs (in quanta, |cs| <= 2^36) into integers
// h, l with h 2^SPLIT + l = rint(cs), |h| <= 2^18, |l| <= 2^17.  Rounding to
// an integer by adding 1.5 * 2^23 is exact for |x| < 2^22; the subtraction
// cs - h 2^SPLIT is exact (Sterbenz).  Only FP32 adds and integer ops, no
// 64-bit conversions.
__device__ inline void split_fix(float cs, int &h, int &l) {
  const float MAGIC = 12582912.0f, MAGIC_H = 3298534883328.0f;  // 1.5 2^23, 1.5 2^41 (ulp 2^SPLIT)
  const float hm = __fadd_rn(cs, MAGIC_H);                        // cs rounded to a multiple of 2^18
  h = __float_as_int(hm) - 0x54400000;
  const float lf = __fsub_rn(cs, __fsub_rn(hm, MAGIC_H));       // exact
  l = __float_as_int(__fadd_rn(lf, MAGIC)) - 0x4B400000;
}

// bilinear interpolation of field c in cell (i, j) at offsets (a, b).  LERP:
// two linear interpolations along i and one along j (six operations, no
// weights); otherwise the four weights, shared by the components that share a
// staggered point (the form the kernels that hold more live values keep: the
// other one makes them spill)
template <bool LERP, class W>
__device__ inline float bilin(const W &w, int c, int i, int j, float a, float b) {
  if (LERP) {
    const float v0 = fmaf(a, w.fld(c, i + 1, j) - w.fld(c, i, j), w.fld(c, i, j));
    const float v1 = fmaf(a, w.fld(c, i + 1, j + 1) - w.fld(c, i, j + 1), w.fld(c, i, j + 1));
    return fmaf(b, v1 - v0, v0);
  }
  return (1.f - a) * (1.f - b) * w.fld(c, i, j) + a * (1.f - b) * w.fld(c, i + 1, j) +
         (1.f - a) * b * w.fld(c, i, j + 1) + a * b * w.fld(c, i + 1, j + 1);
}

// Villasenor-Buneman fluxes of a straight path p -> q inside cell (i, j)
// (local coordinates in [0, 1], Eq. Jcons, Sec. 3.3).  GUARD skips the terms
// of a zero component, which the segments of a split path often have; a zero
// term adds nothing to the exact sums, so either form gives the same bits.
template <bool GUARD = true, class W>
__device__ inline void vb_seg(const W &w, float scale, int i, int j, float p1, float p2, float q1, float q2) {
  const float d1 = q1 - p1, d2 = q2 - p2, m1 = 0.5f * (p1 + q1), m2 = 0.5f * (p2 + q2);
  const float a = scale * d1, b = scale * d2;
  int h, l;
  if (!GUARD || a != 0.f) {
    split_fix(a * (1.f - m2), h, l);
    w.add(0, i, j, h, l);
    split_fix(a * m2, h, l);
    w.add(0, i, j + 1, h, l);
  }
  if (!GUARD || b != 0.f) {
    split_fix(b * (1.f - m1), h, l);
    w.add(1, i, j, h, l);
    split_fix(b * m1, h, l);
    w.add(1, i + 1, j, h, l);
  }
}

// log1p, atan and expm1 for the small arguments of a single step: truncated
// Taylor series (relative truncation s^6/7, t^8/9 and y^6/720: below 1.3e-10
// for |x| < 1/32), otherwise the library functions
// (the _series forms alone when the arguments are known to be small)
__device__ inline float log1p_series(float s) {
  return s * (1.f - s * (0.5f - s * (0.33333334f - s * (0.25f - s * (0.2f - s * 0.16666667f)))));
}
__device__ inline float atan_series(float y, float x) {
  const float t = y * rcp_(x), t2 = t * t;
  return t * (1.f - t2 * (0.33333334f - t2 * (0.2f - t2 * 0.14285715f)));
}
__device__ inline float exp_series(float y) {
  return 1.f + y * (1.f + y * (0.5f + y * (0.16666667f + y * (0.041666668f + y * 0.008333334f))));
}
__device__ inline float log1p_small(float s) { return fabsf(s) < 0.03125f ? log1p_series(s) : log1pf(s); }
__device__ inline float atan2_small(float y, float x) {
  return x > 0.f && fabsf(y) < 0.03125f * x ? atan_series(y, x) : atan2f(y, x);
}
__device__ inline float exp_small(float y) { return fabsf(y) < 0.03125f ? exp_series(y) : expf(y); }

__device__ inline float clamp01(float v) { return fminf(fmaxf(v, 0.f), 1.f); }



// ---- momentum in increments ----------------------------------------------
// The FP32 step computes each change of the momentum -- the push, then the
// rotation into the particle's new local frame -- as an increment du whose
// rounding errors are relative to |du|, not to |u|: for a particle turning by
// a small angle per step they are that much smaller, and the step adds to u
// only the rounding of the one sum u + du that stores it.
//
// This arithmetic is written with explicitly rounded operations: the step is
// inlined twice (shared-memory window and global memory), and a product the
// compiler fused into an FMA in one copy but not in the other would make the
// two paths differ in the last bit.

__device__ __forceinline__ float mul_(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// a x b - c x d (one component of a cross product)
__device__ __forceinline__ float cross_(float a, float b, float c, float d) { return fma_(a, b, -mul_(c, d)); }
__device__ __forceinline__ float dot3_(float a0, float a1, float a2, float b0, float b1, float b2) {
  return fma_(a0, b0, fma_(a1, b1, mul_(a2, b2)));
}
// sin x and cos x - 1 of a small angle: x (1 - x^2/6 + x^4/120) and
// -x^2/2 (1 - x^2/12 + x^4/360), relative truncation below x^6/5040 (under
// 2^-28 for |x| < 0.16)
__device__ __forceinline__ void sin_cosm1_series(float x, float &s, float &cm1) {
  const float x2 = mul_(x, x);
  s = mul_(x, fma_(-x2, fma_(-x2, 0.008333334f, 0.16666667f), 1.f));
  cm1 = mul_(mul_(-0.5f, x2), fma_(-x2, fma_(-x2, 0.0027777778f, 0.083333336f), 1.f));
}

// Vay (2008) push, Sec. 2, as u' - u: with a = u + (q dt/m) E + v x tau and
// t = tau / gamma', u' = s (a + (a.t) t + a x t), s = 1 / (1 + t^2), i.e.
// u' - a = s ((a.t) t + a x t - t^2 a).
__device__ inline void vay_delta(float qmdt, const float E[3], const float B[3], const float u[3], float du[3]) {
  const float h = mul_(0.5f, qmdt);
  const float ig0 = rsqrt_(add_(1.f, dot3_(u[0], u[1], u[2], u[0], u[1], u[2])));
  const float tau0 = mul_(h, B[0]), tau1 = mul_(h, B[1]), tau2 = mul_(h, B[2]);
  const float v0 = mul_(u[0], ig0), v1 = mul_(u[1], ig0), v2 = mul_(u[2], ig0);
  const float d0 = fma_(qmdt, E[0], cross_(v1, tau2, v2, tau1));
  const float d1 = fma_(qmdt, E[1], cross_(v2, tau0, v0, tau2));
  const float d2 = fma_(qmdt, E[2], cross_(v0, tau1, v1, tau0));
  const float a0 = add_(u[0], d0), a1 = add_(u[1], d1), a2 = add_(u[2], d2);
  const float tau2s = dot3_(tau0, tau1, tau2, tau0, tau1, tau2);
  const float ustar = dot3_(a0, a1, a2, tau0, tau1, tau2);
  const float sigma = sub_(add_(1.f, dot3_(a0, a1, a2, a0, a1, a2)), tau2s);
  const float disc = fma_(sigma, sigma, mul_(4.f, fma_(ustar, ustar, tau2s)));
  const float g2 = mul_(0.5f, add_(sigma, sqrtf(disc)));
  const float ig = rsqrt_(g2);
  const float t0 = mul_(tau0, ig), t1 = mul_(tau1, ig), t2 = mul_(tau2, ig);
  const float tt = dot3_(t0, t1, t2, t0, t1, t2);
  const float sc = rcp_(add_(1.f, tt));
  const float at = dot3_(a0, a1, a2, t0, t1, t2);
  du[0] = fma_(sc, sub_(fma_(at, t0, cross_(a1, t2, a2, t1)), mul_(tt, a0)), d0);
  du[1] = fma_(sc, sub_(fma_(at, t1, cross_(a2, t0, a0, t2)), mul_(tt, a1)), d1);
  du[2] = fma_(sc, sub_(fma_(at, t2, cross_(a0, t1, a1, t0)), mul_(tt, a2)), d2);
}

// Boris (1970) push, Sec. 2, as u' - u: half electric kick h E, rotation
// u- -> u+ = u- + (u- + u- x t) x s, half kick; u' - u = 2 h E + (u- + u- x t) x s.
__device__ inline void boris_delta(float qmdt, const float E[3], const float B[3], const float u[3], float du[3]) {
  const float h = mul_(0.5f, qmdt);
  const float he0 = mul_(h, E[0]), he1 = mul_(h, E[1]), he2 = mul_(h, E[2]);
  const float um0 = add_(u[0], he0), um1 = add_(u[1], he1), um2 = add_(u[2], he2);
  const float ig = rsqrt_(add_(1.f, dot3_(um0, um1, um2, um0, um1, um2)));
  const float hi = mul_(h, ig);
  const float t0 = mul_(hi, B[0]), t1 = mul_(hi, B[1]), t2 = mul_(hi, B[2]);
  const float f = mul_(2.f, rcp_(add_(1.f, dot3_(t0, t1, t2, t0, t1, t2))));
  const float p0 = add_(um0, cross_(um1, t2, um2, t1)), p1 = add_(um1, cross_(um2, t0, um0, t2)),
              p2 = add_(um2, cross_(um0, t1, um1, t0));
  const float s0 = mul_(f, t0), s1 = mul_(f, t1), s2 = mul_(f, t2);
  du[0] = fma_(2.f, he0, cross_(p1, s2, p2, s1));
  du[1] = fma_(2.f, he1, cross_(p2, s0, p0, s2));
  du[2] = fma_(2.f, he2, cross_(p0, s1, p1, s0));
}

// Specialisations of the step: the grid maps, pusher and analytic field kind
// fixed at compile time for the two common configurations, so their branches
// fold away (8 % faster than reading them from the arguments), on grids fine
// enough that the radial and meridional series need no general fallback
// (pic_ctx::small_steps); SPEC_GENERIC reads them at run time.
enum Spec { SPEC_GENERIC = 0, SPEC_MONOPOLE = 1, SPEC_ROTATOR = 2 };
template <int SPEC>
struct Flags {
  bool r_log, th_ea;
  int pusher, vacuum;
  __device__ explicit Flags(const Args32 &A)
      : r_log(SPEC == SPEC_GENERIC ? A.r_log != 0 : true),
        th_ea(SPEC == SPEC_GENERIC ? A.th_ea != 0 : SPEC == SPEC_ROTATOR),
        pusher(SPEC == SPEC_GENERIC ? A.pusher : PIC_VAY),
        vacuum(SPEC == SPEC_GENERIC ? A.vacuum : (SPEC == SPEC_ROTATOR ? PIC_VAC_MONOPOLE_ROTATOR : PIC_VAC_MONOPOLE)) {}
};

// One particle step.  Returns false when the particle is removed.
template <int SPEC, class W>
__device__ inline bool step32(const Args32 &A, const W &w, int64_t k, uint32_t &cell, float &dx, float &dy, float &ur,
                              float &ut, float &up, const float qw) {
  const Flags<SPEC> F(A);
  const int ci = (int)(cell >> 16) - CELL_BIAS, cj = (int)(cell & 0xffffu);
  // ---- geometry of the particle's position (Sec. 3.2) -----------------------
  const float rn = w.rad(ci);
  constexpr bool series = SPEC != SPEC_GENERIC;  // arguments below 1/32: no fallback
  const float r = F.r_log ? rn * (series ? exp_series(dx * A.dxi) : exp_small(dx * A.dxi)) : rn + dx * A.dxi;
  // sin and cos of theta from the distance to the nearer pole, which both
  // offsets resolve to FP32 relative precision (1 - x2/nth would cancel)
  const float x2 = (float)cj + dy;                 // distance to the north pole
  const float rest = (float)(A.nth - cj) - dy;     // distance to the south pole
  float st, ct;
  if (F.th_ea) {  // cos th = 1 - 2 x2/nth, sin th = 2 sqrt(x2 (nth - x2))/nth
    ct = (rest - x2) * A.inv_nth;
    st = 2.f * sqrtf(fmaxf(x2 * rest, 0.f)) * A.inv_nth;
  } else if (series) {
    // linear map: the node angle's sine and cosine from the column table,
    // turned by the offset's angle (at most pi / nth, nth >= 32 on the
    // specialised grids: short series).  The node taken is the one on the
    // pole's side of the particle in its hemisphere, so both terms of sin th
    // have one sign and sin th keeps FP32 relative precision up to the poles.
    const bool north = 2 * cj < A.nth;
    const float2 n = w.ang(north ? cj : cj + 1);
    float sb, cb1;
    sin_cosm1_series(mul_(north ? dy : dy - 1.f, A.pi_nth), sb, cb1);
    st = fma_(n.y, sb, fma_(n.x, cb1, n.x));   // sin th_n cos b + cos th_n sin b
    ct = fma_(-n.x, sb, fma_(n.y, cb1, n.y));  // cos th_n cos b - sin th_n sin b
  } else if (x2 <= rest) {
    sincospif(x2 * A.inv_nth, &st, &ct);
  } else {
    sincospif(rest * A.inv_nth, &st, &ct);
    ct = -ct;
  }
  // ---- gather + push (ballistic inside the outer conductor) -----------------
  float du[3] = {0.f, 0.f, 0.f};  // momentum change of the step: push, then frame rotation
  if (ci < A.nr) {
    float E[3], B[3];
    const Vac<float> V{F.vacuum, A.b0, A.r_min, A.omega_t};
    vacuum_field<float>(V, r, st, ct, ci < 0, E, B);
    if (F.vacuum == PIC_VAC_MONOPOLE || F.vacuum == PIC_VAC_MONOPOLE_ROTATOR) {  // monopole B_r = b0 (r0/r)^2 with b0 to ~1e-14
      const float q = A.r_min * rcp_(r);
      B[0] = fmaf(A.b0_lo, q * q, B[0]);
    }
    if (ci >= 0) {  // plasma field only outside the inner conductor
      const bool hx = dx >= 0.5f, hy = dy >= 0.5f;
      const int ih = hx ? ci : ci - 1, jh = hy ? cj : cj - 1;
      const float ah = hx ? dx - 0.5f : dx + 0.5f, bh = hy ? dy - 0.5f : dy + 0.5f;
      constexpr bool L = SPEC == SPEC_MONOPOLE;
      E[0] += bilin<L>(w, ER, ih, cj, ah, dy);
      E[1] += bilin<L>(w, ETH, ci, jh, dx, bh);
      E[2] += bilin<L>(w, EPH, ci, cj, dx, dy);
      B[0] += bilin<L>(w, BR, ci, jh, dx, bh);
      B[1] += bilin<L>(w, BTH, ih, cj, ah, dy);
      B[2] += bilin<L>(w, BPH, ih, jh, ah, bh);
    }
    const float u[3] = {ur, ut, up};
    // local (r, th, ph) is a right-handed orthonormal frame: the Cartesian
    // push formulas apply to its components unchanged
    const float qmdt = qw > 0.f ? A.qmdt : -A.qmdt;
    if (F.pusher == PIC_BORIS) boris_delta(qmdt, E, B, u, du);
    else vay_delta(qmdt, E, B, u, du);
  }
  // u^{n+1/2} in FP32, for the move
  const float pr = add_(ur, du[0]), pt = add_(ut, du[1]), pp = add_(up, du[2]);
  // ---- move in the local frame (Sec. 3.3) -----------------------------------
  const float ig = rsqrt_(1.f + pr * pr + pt * pt + pp * pp);
  const float vr = pr * ig, vt = pt * ig, vp = pp * ig;
  const float Dr = fmaf(vr, A.dt, vr * A.dt_lo), Dt = fmaf(vt, A.dt, vt * A.dt_lo), Dp = fmaf(vp, A.dt, vp * A.dt_lo);
  const float ir = rcp_(r);
  const float a = Dr * ir, b = Dt * ir, c = Dp * ir;
  const float s = a * (2.f + a) + b * b + c * c;  // (r'/r)^2 - 1
  const float L1 = F.r_log ? 0.5f * (series ? log1p_series(s) : log1p_small(s)) : r * s * rcp_(1.f + sqrtf(1.f + s));
  const float D1 = fmaf(L1, A.inv_dxi, L1 * A.inv_dxi_lo);
  const float p = r + Dr, q = Dt;
  const float Px = p * st + q * ct, Pz = p * ct - q * st;  // displaced point, (R, z) before rotating back
  const float Rn = sqrtf(Px * Px + Dp * Dp);
  const float kap = Px >= 0.f ? (Rn + Px > 0.f ? Dp * Dp * rcp_(Rn + Px) : 0.f) : Rn - Px;  // R' - Px
  const float dth = series ? atan_series(q + ct * kap, p + st * kap) : atan2_small(q + ct * kap, p + st * kap);
  // sin(dth) and cos(dth) - 1 of the meridional rotation, from the half angle
  // (or, for the small angles of the specialised grids, short series)
  float D2, sd, cd1;
  if (F.th_ea || !series) {
    float sh, ch;
    sincosf(0.5f * dth, &sh, &ch);
    sd = mul_(2.f, mul_(sh, ch));
    cd1 = mul_(-2.f, mul_(sh, sh));
    D2 = F.th_ea ? A.nth_f * (st * ch + ct * sh) * sh : fmaf(dth, A.k2_hi, dth * A.k2_lo);
  } else {
    sin_cosm1_series(dth, sd, cd1);
    D2 = fmaf(dth, A.k2_hi, dth * A.k2_lo);
  }
  // new cell and offsets (carries are exact integers)
  float tx = dx + D1, ty = dy + D2;
  int kx = (int)floorf(tx), ky = (int)floorf(ty);
  float nx = tx - (float)kx, ny = ty - (float)ky;
  if (nx >= 1.f) { nx = 0.f; ++kx; }
  if (ny >= 1.f) { ny = 0.f; ++ky; }
  int ncj = cj + ky;
  if (ncj < 0) { ncj = 0; ky = -cj; ny = 0.f; }                       // rounding below the axis
  if (ncj > A.nth - 1) { ncj = A.nth - 1; ky = ncj - cj; ny = 1.f; }   // rounding past the south axis
  // momentum into the new local frame, as an increment: Cartesian at phi = 0
  // (x along R), rotated back about z by -phi' (cos phi' - 1 = -kap / R',
  // sin phi' = Dp / R'), then into (r', th') at th' = th + dth:
  //   u_r' = u_r cos dth + u_th sin dth + dx st',  u_th' = -u_r sin dth + u_th cos dth + dx ct',
  //   u_ph' = u_ph + dy,  with (dx, dy) the change of (u_x, u_ph) under the azimuthal rotation
  {
    const float ux = fma_(pr, st, mul_(pt, ct));
    const float iRn = Rn > 0.f ? rcp_(Rn) : 0.f;
    const float cm1 = mul_(-kap, iRn), sph = mul_(Dp, iRn);
    const float dxr = fma_(ux, cm1, mul_(sph, pp)), dyr = fma_(pp, cm1, -mul_(sph, ux));
    const float irn = rsqrtf(fmaxf(fma_(Rn, Rn, mul_(Pz, Pz)), 1e-30f));
    const float stn = mul_(Rn, irn), ctn = mul_(Pz, irn);
    du[0] = add_(du[0], fma_(pr, cd1, fma_(pt, sd, mul_(dxr, stn))));
    du[1] = add_(du[1], fma_(pt, cd1, fma_(-pr, sd, mul_(dxr, ctn))));
    du[2] = add_(du[2], dyr);
  }
  const float nur = add_(ur, du[0]), nut = add_(ut, du[1]), nup = add_(up, du[2]);
  if (!(isfinite(nx) && isfinite(ny) && isfinite(nur) && isfinite(nut) && isfinite(nup)) || kx < -1 || kx > 1 ||
      ky < -1 || ky > 1) {
    atomicOr(A.err, (isfinite(nx) && isfinite(nur)) ? ERR_COURANT : ERR_NAN);
    return false;
  }
  // ---- Villasenor-Buneman deposit along the grid-coordinate path -----------
  // Three segments, split where the path crosses the x and y grid lines in
  // the order it meets them; a line not crossed puts its segment at zero
  // length (zero terms are skipped).  Branch-free, so lanes that cross and
  // lanes that do not run the same instructions -- except for two votes of
  // the converged group: when no lane crosses a line the path is its one
  // nonzero segment (the same terms as in the general form, without the
  // zero-component tests: a zero term adds nothing), and when no lane crosses
  // both lines the third segment is empty for every lane.  Each lane's terms
  // are the same whichever form its group takes.  The move of one step is a small
  // fraction of a cell away from the inner boundary (about 0.35 / r of one at
  // 4096 log cells), so most warps take it there.
  const float scale = qw * w.fs;  // exact: fs is a power of two
  const unsigned grp = __activemask();
  if (__all_sync(grp, (kx | ky) == 0)) {
    vb_seg<false>(w, scale, ci, cj, dx, dy, nx, ny);
  } else {
  const float Dxs = kx == 0 ? nx - dx : (kx > 0 ? (1.f - dx) + nx : -(dx + (1.f - nx)));
  const float Dys = ky == 0 ? ny - dy : (ky > 0 ? (1.f - dy) + ny : -(dy + (1.f - ny)));
  // crossing parameters: any point on the crossed grid line keeps charge
  // conservation exact, so an approximate reciprocal is enough here
  const float sx = kx > 0 ? (1.f - dx) * rcp_(Dxs) : (kx < 0 ? -dx * rcp_(Dxs) : 2.f);
  const float sy = ky > 0 ? (1.f - dy) * rcp_(Dys) : (ky < 0 ? -dy * rcp_(Dys) : 2.f);
  const float Xo = kx > 0 ? 1.f : 0.f, Xn = 1.f - Xo;  // crossed x line in the old / new x frame
  const float Yo = ky > 0 ? 1.f : 0.f, Yn = 1.f - Yo;
  const bool xfirst = sx <= sy;
  // first crossing point, in the frame of the cell the path leaves
  float c1x, c1y;
  if (xfirst) { c1x = kx ? Xo : nx; c1y = kx ? clamp01(dy + sx * Dys) : ny; }
  else        { c1y = Yo; c1x = clamp01(dx + sy * Dxs); }
  // cell of the middle segment and the entry point there
  const int mi = ci + (xfirst ? kx : 0), mj = cj + (xfirst ? 0 : ky);
  const float e1x = (xfirst && kx) ? Xn : c1x, e1y = (!xfirst) ? Yn : c1y;
  vb_seg(w, scale, ci, cj, dx, dy, c1x, c1y);
  if (__all_sync(grp, (kx & ky) == 0)) {
    // no lane of the group crosses both lines (kx & ky is nonzero only when
    // both are): the middle segment ends at the end point and the third has
    // zero length, as in the general form below
    vb_seg(w, scale, mi, mj, e1x, e1y, nx, ny);
  } else {
  // second crossing point, in the frame of the middle cell
  float c2x, c2y;
  if (kx && ky) {
    if (xfirst) { c2y = Yo; c2x = clamp01(nx - (1.f - sy) * Dxs); }
    else        { c2x = Xo; c2y = clamp01(ny - (1.f - sx) * Dys); }
  } else {
    c2x = nx; c2y = ny;
  }
  const float e2x = (kx && ky && !xfirst) ? Xn : c2x, e2y = (kx && ky && xfirst) ? Yn : c2y;
  vb_seg(w, scale, mi, mj, e1x, e1y, c2x, c2y);
  vb_seg(w, scale, ci + kx, cj + ky, e2x, e2y, nx, ny);
  }
  }
  // azimuthal flux: charge crossing the meridional half-plane, qw dphi / 2 pi,
  // area weights at the midpoint of the grid path
  {
    float phi = atan2_small(Dp, Px);
    if (Px < 0.f && pp * pp <= (float)(AXIS_TIE * AXIS_TIE) * (pr * pr + pt * pt + pp * pp))
      phi = axis_tie(A.ties, A.ids[k], phi);  // rare: see AxisTies
    const float v = scale * phi * 0.15915494309189535f;
    const float mx = 0.5f * (dx + (float)kx + nx), my = 0.5f * (dy + (float)ky + ny);
    const float fx = floorf(mx), fy = floorf(my);
    const float wx = mx - fx, wy = my - fy;
    const int i0 = ci + (int)fx, j0 = cj + (int)fy;
    {  // v is nonzero for nearly every particle: no test
      int h, l;
      split_fix(v * (1.f - wx) * (1.f - wy), h, l);
      w.add(2, i0, j0, h, l);
      split_fix(v * wx * (1.f - wy), h, l);
      w.add(2, i0 + 1, j0, h, l);
      split_fix(v * (1.f - wx) * wy, h, l);
      w.add(2, i0, j0 + 1, h, l);
      split_fix(v * wx * wy, h, l);
      w.add(2, i0 + 1, j0 + 1, h, l);
    }
  }
  // ---- store; removal once the filtered shape is inside a conductor ---------
  const int nci = ci + kx;
  if (nci < -(A.n_filt + 1) || nci >= A.nr + A.n_filt + 1) return false;
  cell = ((uint32_t)(nci + CELL_BIAS) << 16) | (uint32_t)ncj;
  dx = nx; dy = ny; ur = nur; ut = nut; up = nup;
  return true;
}

// the rare path: a particle outside its tile's window (inlined: an
// out-of-line call costs register spills around it in the hot loop)
template <int SPEC>
__device__ inline bool step32_global(const Args32 &A, float fs, int64_t k, uint32_t &cell, float &dx, float &dy,
                                     float &ur, float &ut, float &up, const float qw) {
  const GlobAcc gw{&A, fs};
  return step32<SPEC>(A, gw, k, cell, dx, dy, ur, ut, up, qw);
}

template <int SPEC, class SW>
__device__ inline void process_v(const Args32 &A, Parts32 P, int64_t k, bool win, const SW &sw,
                                 int wi_lo, int wi_hi, int wj_lo, int wj_hi, int &dead, const float qw,
                                 uint32_t cell, float dx, float dy, float ur, float ut, float up) {
  if (qw == 0.f) return;
  const int ci = (int)(cell >> 16) - CELL_BIAS, cj = (int)(cell & 0xffffu);
  bool alive;
  if (win && ci >= wi_lo && ci < wi_hi && cj >= wj_lo && cj < wj_hi)
    alive = step32<SPEC>(A, sw, k, cell, dx, dy, ur, ut, up, qw);
  else
    alive = step32_global<SPEC>(A, sw.fs, k, cell, dx, dy, ur, ut, up, qw);
  if (!alive) { P.qw[k] = 0.f; ++dead; return; }
  P.cell[k] = cell;
  P.dx[k] = dx; P.dy[k] = dy;
  P.ur[k] = ur; P.ut[k] = ut; P.up[k] = up;
}

template <int SPEC, class SW>
__device__ inline void process(const Args32 &A, Parts32 P, int64_t k, bool win, const SW &sw,
                               int wi_lo, int wi_hi, int wj_lo, int wj_hi, int &dead) {
  process_v<SPEC>(A, P, k, win, sw, wi_lo, wi_hi, wj_lo, wj_hi, dead, P.qw[k], P.cell[k], P.dx[k], P.dy[k], P.ur[k],
                  P.ut[k], P.up[k]);
}


// ---- the field window through the tensor memory accelerator ---------------
// Each FP32 field is a 2-D tensor (LD columns x rows of the padded grid).  A
// tile's window (WI rows x WJ columns from (wi0, wj0)) is fetched as one box
// per field whose first column is wj0 - WOFF: with the padding PJ a multiple of
// 8 and every tile's j0 a multiple of 8, that column is a multiple of 4 floats
// (16 bytes), as a tiled copy requires; the box is WB columns wide, a whole
// number of 16-byte units.  The boxes land in a staging area, are laid out at
// the window's own pitch WJ (odd, so lanes in different rows fall in different
// banks) and the staging area then becomes the deposit accumulators.
constexpr int WOFF = 3;
static_assert((PAD - H - 1 - WOFF) % 8 == 0, "window box column must stay 16-byte aligned");
template <int TI, int TJ>
struct Box {
  static constexpr int WI = Win<TI, TJ>::WI, WJ = Win<TI, TJ>::WJ, WN = Win<TI, TJ>::WN;
  static constexpr int WB = (WOFF + WJ + 3) / 4 * 4;        // box width (floats)
  static constexpr int SLOT = (WI * WB + 31) / 32 * 32;     // one field's box, 128-byte multiple
  static constexpr int SF = (6 * WN + 31) / 32 * 32;        // laid-out window (floats)
  static constexpr int U = 6 * SLOT > 6 * WN ? 6 * SLOT : 6 * WN;  // staging, then accumulators
};

struct TileMaps {  // the six field tensors for the current tile shape (kernel parameter)
  CUtensorMap m[6];
};

__device__ inline uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// per-thread asynchronous copy of 4 bytes global -> shared (no registers held)
__device__ inline void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ inline void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ inline void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ inline void tma_window(float *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// wait for phase 0 of the window barrier, at most `limit` polls
__device__ inline bool window_wait(uint64_t *bar, long long limit) {
  for (long long k = 0; k < limit; ++k) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar))
        : "memory");
    if (done) return true;
  }
  return false;
}

// Self-test of the bounded wait above: thread 0 of a one-warp block arms an
// mbarrier for 16 bytes that no copy will deliver (arrive_first = 0) or
// completes its phase itself first (arrive_first = 1), then waits at most
// `limit` polls; on giving up it sets ERR_TIMEOUT, as the tile kernel does.
// Nothing is in flight, so the block can leave after a timeout.
__global__ void k_wait_selftest(long long limit, int arrive_first, int *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (arrive_first) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
  } else {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar)), "r"(16u) : "memory");
  }
  if (!window_wait(&bar, limit)) atomicOr(err, ERR_TIMEOUT);
}

// Tensor maps read by the TMA unit from global memory (the batched ensemble
// kernel's per-member maps, written by a host copy before any launch) are
// ordered after those writes by an acquire fence of the tensor-map proxy.
__device__ inline void tensormap_acquire(const CUtensorMap *map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

// One tile CTA (or one block of unbinned particles) of the FP32 step: block
// `blk` of the member whose arguments are A and P, its six field tensor maps
// at `maps` (kernel parameters, or global memory when GMAPS).
template <int TI, int TJ, int SPEC, bool GMAPS>
__device__ __forceinline__ void tiles32_block(const Args32 &A, const Parts32 &P, const CUtensorMap *maps,
                                              unsigned blk) {
  using BX_ = Box<TI, TJ>;
  constexpr int WI = BX_::WI, WJ = BX_::WJ, WN = BX_::WN, WB = BX_::WB, SLOT = BX_::SLOT;
  __shared__ __align__(128) float sbuf[BX_::SF + BX_::U];
  __shared__ __align__(16) uint32_t spf[2][7][NT];  // each thread's next particle, copied ahead
  float *const sf = sbuf;                                      // 6 WN: the window
  float *const stage = sbuf + BX_::SF;                         // 6 SLOT: the boxes, first
  int *const shi = reinterpret_cast<int *>(sbuf + BX_::SF);    // 3 WN: then the accumulators
  int *const slo = shi + 3 * WN;                               // 3 WN
  __shared__ float srn[WI];
  __shared__ float2 stn[WJ];
  __shared__ int sdead, sok;
  __shared__ __align__(8) uint64_t sbar;
  int dead = 0;
  const float fs = __int_as_float((127 + KFIX - qexp_value(A.qexp)) << 23);  // 2^(KFIX - e)
  if (blk < (uint64_t)A.nunits) {
    const long long u = A.units[blk];
    const int t = (int)(u >> 32);
    const int64_t b0 = A.start[(int64_t)t * A.tc] + (u & 0xffffffffll) * A.unit;
    const int64_t b1 = min(A.start[(int64_t)(t + 1) * A.tc], b0 + A.unit);
    if (b1 <= b0) return;
    const int i0 = A.row0 + (t / A.ntj) * TI, j0 = (t % A.ntj) * TJ;
    const int wi0 = i0 - H - 1, wj0 = j0 - H - 1;
    if (threadIdx.x == 0) {
      sdead = 0;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sbar)));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&sbar)),
                   "r"((uint32_t)(6 * WI * WB * sizeof(float)))
                   : "memory");
      const int x = wj0 - WOFF + A.PJ, y = wi0 + A.PI;  // x: a multiple of 4 (static_assert above)
      if (GMAPS) {
#pragma unroll
        for (int c = 0; c < 6; ++c) tensormap_acquire(maps + c);
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) tma_window(stage + c * SLOT, maps + c, x, y, &sbar);
      // bounded wait: on a timeout the error is latched, the copies get a
      // second bounded wait (they write into this block's shared memory) and
      // the tile is skipped
      bool ok = window_wait(&sbar, 1ll << 26);
      if (!ok) {
        atomicOr(A.err, ERR_TIMEOUT);
        window_wait(&sbar, 1ll << 26);
      }
      sok = ok ? 1 : 0;
    }
    for (int e = threadIdx.x; e < WI; e += NT) srn[e] = A.r_n[wi0 + e + A.PI];
    if (SPEC != SPEC_GENERIC)
      for (int e = threadIdx.x; e < WJ; e += NT) stn[e] = A.th_n[wj0 + e + A.PJ];
    __syncthreads();
    if (!sok) return;
    for (int e = threadIdx.x; e < WN; e += NT) {
      const int r = e / WJ, q = e % WJ;
#pragma unroll
      for (int c = 0; c < 6; ++c) sf[c * WN + e] = stage[c * SLOT + r * WB + q + WOFF];
    }
    __syncthreads();  // the staging area becomes the accumulators
    for (int e = threadIdx.x; e < 3 * WN; e += NT) { shi[e] = 0; slo[e] = 0; }
    __syncthreads();
    const SmemAcc<WJ, WN> sw{sf, shi, slo, srn, stn, wi0, wj0, fs};
    {
      const int t = threadIdx.x;
      auto fetch = [&](int buf, int64_t k) {
        cp_async4(&spf[buf][0][t], P.qw + k); cp_async4(&spf[buf][1][t], P.cell + k);
        cp_async4(&spf[buf][2][t], P.dx + k); cp_async4(&spf[buf][3][t], P.dy + k);
        cp_async4(&spf[buf][4][t], P.ur + k); cp_async4(&spf[buf][5][t], P.ut + k);
        cp_async4(&spf[buf][6][t], P.up + k);
      };
      int64_t k = b0 + t;
      if (k < b1) fetch(0, k);
      cp_commit();
      for (int buf = 0; k < b1; k += NT, buf ^= 1) {
        if (k + NT < b1) fetch(buf ^ 1, k + NT);
        cp_commit();
        cp_wait<1>();  // this particle's copies (the next one's may still be in flight)
        process_v<SPEC>(A, P, k, true, sw, i0 - H, i0 + TI + H, j0 - H, j0 + TJ + H, dead,
                        __uint_as_float(spf[buf][0][t]), spf[buf][1][t], __uint_as_float(spf[buf][2][t]),
                        __uint_as_float(spf[buf][3][t]), __uint_as_float(spf[buf][4][t]),
                        __uint_as_float(spf[buf][5][t]), __uint_as_float(spf[buf][6][t]));
      }
      cp_wait<0>();
    }
    if (dead) atomicAdd(&sdead, dead);
    __syncthreads();
    for (int e = threadIdx.x; e < WN; e += NT) {
      const size_t o = pidx(A, wi0 + e / WJ, wj0 + e % WJ);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int hsum = shi[c * WN + e], lsum = slo[c * WN + e];
        if (abs(hsum) >= (1 << 30) || abs(lsum) >= (1 << 30)) atomicOr(A.err, ERR_CAPACITY);  // near the limit
        const long long v = ((long long)hsum << SPLIT) + (long long)lsum;
        if (v) atomicAdd(reinterpret_cast<unsigned long long *>(A.acc[c] + o), (unsigned long long)v);
      }
    }
    if (threadIdx.x == 0 && sdead) add_ll(A.cnt + CNT_DELETED, sdead);
  } else {  // particles outside any bin (injected since the last sort)
    const SmemAcc<WJ, WN> none{nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0, fs};
    const int64_t k = A.sorted_end + (int64_t)(blk - A.nunits) * NT + threadIdx.x;
    if (k < A.n_used) process<SPEC>(A, P, k, false, none, 0, 0, 0, 0, dead);
    if (dead) add_ll(A.cnt + CNT_DELETED, dead);
  }
}

template <int TI, int TJ, int SPEC>
__global__ void __launch_bounds__(NT, 4) k_tiles32(Args32 A, Parts32 P, const __grid_constant__ TileMaps maps) {
  tiles32_block<TI, TJ, SPEC, false>(A, P, maps.m, blockIdx.x);
}

// One member of a batched launch: its step's arguments and its six field
// tensor maps (device memory) for its tile shape.
struct EnsTileArg {
  Args32 A;
  Parts32 P;
  const CUtensorMap *maps;
};

// Up to ENS_TILE_SLOTS members in one launch, passed as kernel parameters:
// the arguments sit in the same immutable parameter memory as those of
// k_tiles32, so the compiler treats them alike (loads it may hoist out of the
// particle loop), which keeps every member's arithmetic bit-identical to its
// own k_tiles32 launch.  Member k owns blocks [off[k], off[k + 1]).
constexpr int ENS_TILE_SLOTS = 48;
struct EnsTileBatch {
  EnsTileArg a[ENS_TILE_SLOTS];
  int off[ENS_TILE_SLOTS + 1];
  int n;
};
static_assert(sizeof(EnsTileBatch) <= 32000, "kernel parameters are limited to 32 KB");

// the tile kernel over several members of an ensemble in one grid
template <int TI, int TJ, int SPEC>
__global__ void __launch_bounds__(NT, 4) k_ens_tiles32(const __grid_constant__ EnsTileBatch B) {
  int lo = 0, hi = B.n - 1;  // the member owning this block
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((unsigned)B.off[mid] <= blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const EnsTileArg &T = B.a[lo];
  tiles32_block<TI, TJ, SPEC, true>(T.A, T.P, T.maps, blockIdx.x - (unsigned)B.off[lo]);
}

// (double)v * 2^s built on the integer pipes: v rounded to 53 bits (to
// nearest, ties to even, as the FP64 conversion does; exact for the sums
// below 2^53 that occur in practice) and the power of two added to the
// exponent, which is exact while the result stays normal (s in [-126, 64] here).
// The same IEEE value as the conversion and multiply, without the FP64 pipe,
// whose rate on this part made the conversion pass compute-bound.
__device__ inline double fixed_to_f64(long long v, int s) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long m = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  int e = 63 - __clzll((long long)m);  // m in [2^e, 2^(e+1))
  unsigned long long mant;
  if (e <= 52) {
    mant = m << (52 - e);
  } else {
    const int sh = e - 52;
    const unsigned long long q = m >> sh, rem = m & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    mant = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
    if (mant >> 53) { mant >>= 1; ++e; }
  }
  const unsigned long long bits = sign | ((unsigned long long)(e + s + 1023) << 52) | (mant & ((1ull << 52) - 1ull));
  return __longlong_as_double((long long)bits);
}

// fixed point -> FP64 fluxes over the ghost band; clears the accumulators
// (node i, j of the band -g <= i <= nr + g, 0 <= j <= nth)
__device__ __forceinline__ void flux_node(int i, int j, int nr, int nth, int g, int PI, int LD, int PJ,
                                          const long long *qexp, long long *a0, long long *a1, long long *a2,
                                          double *F0, double *F1, double *F2) {
  if (i > nr + g || j > nth) return;
  const int s = qexp_value(qexp) - KFIX;  // one flux unit is 2^s of charge
  const size_t o = (size_t)(i + PI) * LD + (size_t)(j + PJ);
  F0[o] = fixed_to_f64(a0[o], s); a0[o] = 0;
  F1[o] = fixed_to_f64(a1[o], s); a1[o] = 0;
  F2[o] = fixed_to_f64(a2[o], s); a2[o] = 0;
}

__global__ void k_flux_from_acc(int nr, int nth, int g, int PI, int PJ, int LD, const long long *qexp,
                                long long *a0, long long *a1, long long *a2, double *F0, double *F1, double *F2) {
  flux_node(-g + (int)(blockIdx.y * 8 + threadIdx.y), blockIdx.x * 32 + threadIdx.x, nr, nth, g, PI, LD, PJ, qexp,
            a0, a1, a2, F0, F1, F2);
}

// the same over the members of an ensemble: 256-thread blocks, each member's
// band covered by 32 x 8 node blocks as above
__global__ void k_ens_flux(const EnsFieldArg *__restrict__ tab, EnsList L) {
  const int2 e = L.blk[blockIdx.x];
  const EnsFieldArg &E = tab[e.x];
  const Grid &G = E.G;
  const unsigned b = (unsigned)e.y, gx = (unsigned)(G.nth + 1 + 31) / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  flux_node(-G.g + (int)((b / gx) * 8 + ty), (int)((b % gx) * 32 + tx), G.nr, G.nth, G.g, G.PI, G.LD, G.PJ,
            E.qexp, E.acc[0], E.acc[1], E.acc[2], E.Fin[0], E.Fin[1], E.Fin[2]);
}

// ---- counting sort into tile bins (drops removed particles) ---------------
// Bins are numbered cell by cell, tile-major: key = tile * tc + cell index
// inside the tile; removed particles go to the last bin, ntiles * tc.  Keys
// fit in 32 bits: at most (nr + 2g + TI) (nth + TJ) cells with nr, nth <= 32000.
// Two kinds of sort share the bins:
//  - mixing (after particles are loaded or the tile shape changes): by cell,
//    each tile's bin stored transposed (transposed_slot below), so the lanes
//    of a warp step particles of different cells;
//  - keeping (every later sort): by tile only (all of a tile's particles in
//    bin tile * tc), each tile's particles in their previous relative order,
//    which keeps them mixed: particles move a few cells between sorts.
__device__ inline int cell_key(const Args32 &A, uint32_t cell, float qw) {
  if (qw == 0.f) return A.ntiles * A.tc;
  const int ci = (int)(cell >> 16) - CELL_BIAS - A.row0, cj = (int)(cell & 0xffffu);
  const int tile = ((ci / A.ti) * A.ntj + cj / A.tj) * A.tc;
  return A.mix ? tile + (ci % A.ti) * A.tj + cj % A.tj : tile;
}

__device__ __forceinline__ void hist_block(const Args32 &A, const Parts32 &P, int64_t n, int64_t *count,
                                           unsigned blk) {
  const int64_t k = blk * (int64_t)blockDim.x + threadIdx.x;
  const int key = k < n ? cell_key(A, P.cell[k], P.qw[k]) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  if (key >= 0 && lane == __ffs(peers) - 1)
    atomicAdd(reinterpret_cast<unsigned long long *>(count + key), (unsigned long long)__popc(peers));
}

__global__ void k_hist(Args32 A, Parts32 P, int64_t n, int64_t *count) { hist_block(A, P, n, count, blockIdx.x); }

// exclusive scan of nb counts by one block of 1024 threads (the top level of
// the scan below); count becomes the cursor and start[nb] the total
__device__ __forceinline__ void scan_bins_block(int64_t *count, int64_t *start, int nb) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int per = (nb + 1023) / 1024, a = t * per, b = min(nb, a + per);
  int64_t s = 0;
  for (int k = a; k < b; ++k) s += count[k];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int64_t v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t run = part[t] - s;
  for (int k = a; k < b; ++k) {
    const int64_t c = count[k];
    start[k] = run;
    count[k] = run;
    run += c;
  }
  if (t == 1023) start[nb] = part[1023];
}

__global__ void k_scan_bins(int64_t *count, int64_t *start, int nb) { scan_bins_block(count, start, nb); }

// block sum of 256 values (all threads get it)
__device__ inline int64_t block_sum256(int64_t v, int64_t *sm) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  int64_t t = 0;
  for (int w = 0; w < 8; ++w) t += sm[w];
  __syncthreads();
  return t;
}

// multi-block exclusive scan over nb bins, SCAN_CHUNK bins per block of 256
// threads: sums of each chunk, a one-block scan of the sums, then each chunk
// scanned from its offset (16 consecutive bins per thread)
__device__ __forceinline__ void scan_sums_block(const int64_t *count, int64_t nb, int64_t *sums, unsigned blk) {
  __shared__ int64_t sm[8];
  const int64_t a = blk * (int64_t)SCAN_CHUNK;
  int64_t s = 0;
  for (int k = threadIdx.x; k < SCAN_CHUNK; k += 256)
    if (a + k < nb) s += count[a + k];
  s = block_sum256(s, sm);
  if (threadIdx.x == 0) sums[blk] = s;
}

__global__ void k_scan_sums(const int64_t *count, int64_t nb, int64_t *sums) {
  scan_sums_block(count, nb, sums, blockIdx.x);
}

__device__ __forceinline__ void scan_apply_block(int64_t *count, int64_t *start, int64_t nb, const int64_t *offs,
                                                 int nblk, unsigned blk) {
  __shared__ int64_t sm[8];
  const int64_t a = blk * (int64_t)SCAN_CHUNK + threadIdx.x * 16;
  int64_t v[16], s = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) { v[i] = a + i < nb ? count[a + i] : 0; s += v[i]; }
  // exclusive scan of the 256 thread sums
  int64_t x = s;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[w] = x;
  __syncthreads();
  int64_t base = offs[blk];
  for (int k = 0; k < w; ++k) base += sm[k];
  int64_t run = base + x - s;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    if (a + i < nb) { start[a + i] = run; count[a + i] = run; }
    run += v[i];
  }
  if (blk == 0 && threadIdx.x == 0) start[nb] = offs[nblk];
}

__global__ void k_scan_apply(int64_t *count, int64_t *start, int64_t nb, const int64_t *offs, int nblk) {
  scan_apply_block(count, start, nb, offs, nblk, blockIdx.x);
}

// work units of each tile: ceil(n_t / unit), none for an empty tile
__device__ __forceinline__ void unit_count_at(int t, const int64_t *start, int tc, int ntiles, int64_t unit,
                                              int64_t *ucount) {
  if (t >= ntiles) return;
  const int64_t n = start[(int64_t)(t + 1) * tc] - start[(int64_t)t * tc];
  ucount[t] = (n + unit - 1) / unit;
}

__global__ void k_unit_count(const int64_t *start, int tc, int ntiles, int64_t unit, int64_t *ucount) {
  unit_count_at(blockIdx.x * blockDim.x + threadIdx.x, start, tc, ntiles, unit, ucount);
}

// the unit list from the exclusive scan of the counts (uoff[ntiles] = total)
__device__ __forceinline__ void unit_fill_at(int t, const int64_t *uoff, int ntiles, long long *units) {
  if (t >= ntiles) return;
  for (int64_t u = uoff[t]; u < uoff[t + 1]; ++u) units[u] = ((long long)t << 32) | (long long)(u - uoff[t]);
}

__global__ void k_unit_fill(const int64_t *uoff, int ntiles, long long *units) {
  unit_fill_at(blockIdx.x * blockDim.x + threadIdx.x, uoff, ntiles, units);
}

// Order inside a tile's bin.  The counting sort yields the tile's particles
// cell by cell; they are stored transposed: the cell-ordered sequence fills
// the columns of a matrix with TRW columns, and the bin holds its rows.  The
// 32 lanes of a warp, which step consecutive slots, then hold particles about
// n / TRW apart in cell order: different cells, so their deposits rarely hit
// the same shared-memory address in one instruction.  (The results do not
// depend on the order: the deposit sums are exact.)  q: position in cell
// order, n: particles in the bin; returns the slot.
constexpr int TRW = 16;
__device__ inline int64_t transposed_slot(int64_t q, int64_t n) {
  const int64_t R = (n + TRW - 1) / TRW;  // rows
  const int64_t L = n - (R - 1) * TRW;    // columns of R elements; the others hold R - 1
  int64_t c, r;
  if (q < L * R) { c = q / R; r = q - c * R; }
  else { const int64_t u = q - L * R; c = L + u / (R - 1); r = u - (c - L) * (R - 1); }
  return r * TRW + c;
}

__device__ __forceinline__ void scatter_block(const Args32 &A, const Parts32 &S, const Parts32 &D, int64_t n,
                                              int64_t *cursor, unsigned blk) {
  const int64_t k = blk * (int64_t)blockDim.x + threadIdx.x;
  const int trash = A.ntiles * A.tc;
  // every load issued before the cursor atomic, whose round trip they overlap
  const int64_t kk = k < n ? k : 0;
  const uint32_t cell = S.cell[kk];
  const float dx = S.dx[kk], dy = S.dy[kk], ur = S.ur[kk], ut = S.ut[kk], up = S.up[kk], qw = S.qw[kk];
  const int64_t id = S.id[kk];
  const int key = k < n ? cell_key(A, cell, qw) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31, leader = __ffs(peers) - 1;
  unsigned long long base = 0;
  if (key >= 0 && key < trash && lane == leader)
    base = atomicAdd(reinterpret_cast<unsigned long long *>(cursor + key), (unsigned long long)__popc(peers));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (key < 0 || key >= trash) return;
  int64_t d = (int64_t)base + __popc(peers & ((1u << lane) - 1u));
  if (A.mix) {
    const int t = key / A.tc;
    const int64_t t0 = A.start[(int64_t)t * A.tc], t1 = A.start[(int64_t)(t + 1) * A.tc];
    d = t0 + transposed_slot(d - t0, t1 - t0);
  }
  D.cell[d] = cell; D.dx[d] = dx; D.dy[d] = dy;
  D.ur[d] = ur; D.ut[d] = ut; D.up[d] = up;
  D.qw[d] = qw; D.id[d] = id;
}

__global__ void k_scatter_cells(Args32 A, Parts32 S, Parts32 D, int64_t n, int64_t *cursor) {
  scatter_block(A, S, D, n, cursor, blockIdx.x);
}

// ---- the tile sort of several ensemble members at once ---------------------
// One member's sort as the batched kernels read it (device table): the same
// arrays and the same kernel bodies as sort32, every phase one launch for all
// members due, and one read-back of their live counts, unit counts and error
// words.
struct EnsSortArg {
  Args32 A;                   // keys and tile geometry; A.mix: this sort's order
  Parts32 S, D;               // particles before and after the sort
  int64_t n;                  // particles before the sort
  int64_t *count, *start, *bsum;
  int64_t nbins;
  int nblk, ublk, ntiles, tc;
  int64_t *ucount, *usum;
  long long *units;
  int64_t unit;
  const int *err;
  int64_t *out;               // live, units, error bits (for the host)
};

__global__ void k_ens_sort_zero(const EnsSortArg *__restrict__ tab, EnsList L) {
  const int2 e = L.blk[blockIdx.x];
  const EnsSortArg &E = tab[e.x];
  const int64_t q = (int64_t)e.y * blockDim.x + threadIdx.x;
  if (q <= E.nbins) E.count[q] = 0;
}
__global__ void k_ens_hist(const EnsSortArg *__restrict__ tab, EnsList L) {
  const int2 e = L.blk[blockIdx.x];
  const EnsSortArg &E = tab[e.x];
  hist_block(E.A, E.S, E.n, E.count, (unsigned)e.y);
}
// units = 0: the scan of the bin counts; 1: of the per-tile unit counts
__global__ void k_ens_scan_sums(const EnsSortArg *__restrict__ tab, EnsList L, int units) {
  const int2 e = L.blk[blockIdx.x];
  const EnsSortArg &E = tab[e.x];
  if (units) scan_sums_block(E.ucount, E.ntiles, E.usum, (unsigned)e.y);
  else scan_sums_block(E.count, E.nbins, E.bsum, (unsigned)e.y);
}
__global__ void k_ens_scan_bins(const EnsSortArg *__restrict__ tab, EnsList L, int units) {
  const EnsSortArg &E = tab[L.blk[blockIdx.x].x];
  if (units) scan_bins_block(E.usum, E.usum + E.ublk + 1, E.ublk);
  else scan_bins_block(E.bsum, E.bsum + E.nblk + 1, E.nblk);
}
__global__ void k_ens_scan_apply(const EnsSortArg *__restrict__ tab, EnsList L, int units) {
  const int2 e = L.blk[blockIdx.x];
  const EnsSortArg &E = tab[e.x];
  if (units) scan_apply_block(E.ucount, E.ucount, E.ntiles, E.usum + E.ublk + 1, E.ublk, (unsigned)e.y);
  else scan_apply_block(E.count, E.start, E.nbins, E.bsum + E.nblk + 1, E.nblk, (unsigned)e.y);
}
__global__ void k_ens_scatter(const EnsSortArg *__restrict__ tab, EnsList L) {
  const int2 e = L.blk[blockIdx.x];
  const EnsSortArg &E = tab[e.x];
  scatter_block(E.A, E.S, E.D, E.n, E.count, (unsigned)e.y);
}
__global__ void k_ens_unit_count(const EnsSortArg *__restrict__ tab, EnsList L) {
  const int2 e = L.blk[blockIdx.x];
  const EnsSortArg &E = tab[e.x];
  unit_count_at(e.y * blockDim.x + threadIdx.x, E.start, E.tc, E.ntiles, E.unit, E.ucount);
}
__global__ void k_ens_unit_fill(const EnsSortArg *__restrict__ tab, EnsList L) {
  const int2 e = L.blk[blockIdx.x];
  const EnsSortArg &E = tab[e.x];
  unit_fill_at(e.y * blockDim.x + threadIdx.x, E.ucount, E.ntiles, E.units);
}
__global__ void k_ens_sort_out(const EnsSortArg *__restrict__ tab, int m) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const EnsSortArg &E = tab[k];
  E.out[0] = E.start[(int64_t)E.ntiles * E.tc];
  E.out[1] = E.ucount[E.ntiles];
  E.out[2] = *E.err;
}

__global__ void k_charge32(int PI, int PJ, int LD, Parts32 P, int64_t n, double *Q, double *Qa) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double q = P.qw[k];
  if (q == 0.0) return;
  const uint32_t c = P.cell[k];
  const int ci = (int)(c >> 16) - CELL_BIAS, cj = (int)(c & 0xffffu);
  const double w1 = P.dx[k], w2 = P.dy[k];
  const size_t o = (size_t)(ci + PI) * LD + (size_t)(cj + PJ);
  const double c00 = (1 - w1) * (1 - w2), c10 = w1 * (1 - w2), c01 = (1 - w1) * w2, c11 = w1 * w2;
  atomicAdd(Q + o, q * c00); atomicAdd(Q + o + LD, q * c10);
  atomicAdd(Q + o + 1, q * c01); atomicAdd(Q + o + LD + 1, q * c11);
  const double aq = fabs(q);
  atomicAdd(Qa + o, aq * c00); atomicAdd(Qa + o + LD, aq * c10);
  atomicAdd(Qa + o + 1, aq * c01); atomicAdd(Qa + o + LD + 1, aq * c11);
}

__global__ void k_reduce32(Parts32 P, int64_t n, double qm, double *acc, long long *live) {
  double kin = 0.0, ch = 0.0;
  long long l = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const float q = P.qw[k];
    if (q == 0.f) continue;
    const float a = P.ur[k], b = P.ut[k], c = P.up[k], u2 = a * a + b * b + c * c;
    // each particle's (gamma - 1) |qw| in FP32 (gamma - 1 = u^2 / (1 + gamma): no
    // cancellation), summed in FP64; FP64 square roots would make this diagnostic
    // FP64-bound on this part
    kin += (double)(fabsf(q) * (u2 / (1.f + sqrtf(1.f + u2))));
    ch += q;
    l += 1;
  }
  block_sum3(kin / qm, ch, l, acc + ACC_KIN, acc + ACC_CHARGE, live);
}

Args32 make_args(pic_ctx *c, double t) {
  const Grid &G = c->G;
  Args32 A;
  A.nr = G.nr; A.nth = G.nth; A.n_filt = G.n_filt; A.PI = G.PI; A.PJ = G.PJ; A.LD = G.LD;
  A.r_log = G.r_map == PIC_R_LOG; A.th_ea = G.th_map == PIC_TH_EQUAL_AREA;
  A.vacuum = G.vacuum; A.pusher = G.pusher;
  A.dxi = (float)G.dxi; A.inv_dxi = (float)(1.0 / G.dxi); A.dt = (float)G.dt; A.qm = (float)G.qm;
  A.dt_lo = (float)(G.dt - (double)A.dt);
  A.inv_dxi_lo = (float)(1.0 / G.dxi - (double)A.inv_dxi);
  A.k2_hi = (float)(G.nth / M_PI);
  A.k2_lo = (float)(G.nth / M_PI - (double)A.k2_hi);
  A.inv_nth = (float)(1.0 / G.nth); A.nth_f = (float)G.nth;
  A.qexp = c->qexp;
  A.ids = c->p32.id;
  A.ties = axis_ties(c);
  A.r_n = c->r_n32;
  A.th_n = c->th_n32;
  A.pi_nth = (float)(M_PI / G.nth);
  for (int k = 0; k < 6; ++k) A.f[k] = c->f32[k];
  for (int k = 0; k < 3; ++k) A.acc[k] = c->acc[k];
  A.err = c->d_err;
  A.cnt = c->d_cnt;
  A.row0 = c->tiles.row0; A.ntj = c->tiles.ntj; A.ntiles = c->tiles.ntiles;
  // Particles keep whole-grid rows in their packed cell.  A radial slab
  // (rows i0.. of a grid of nr_glob rows) indexes its arrays through a
  // padding offset shifted by i0, tests the conductors and removal against
  // the whole grid and places its tiles at its own rows; a whole grid has
  // i0 = 0 and nr_glob = nr, i.e. these are its own values.
  A.nr = G.nr_glob;
  A.PI = G.PI - G.i0;
  A.row0 = c->tiles.row0 + G.i0;
  A.ti = c->tiles.TI; A.tj = c->tiles.TJ; A.tc = c->tiles.tc;
  A.mix = 0;
  A.start = c->tiles.start;
  A.units = c->tiles.units;
  A.nunits = c->tiles.nunits;
  A.unit = c->tiles.unit;
  A.sorted_end = c->tiles.sorted_end;
  A.n_used = c->n_used;
  A.b0 = (float)G.b0; A.r_min = (float)G.r_min;
  A.b0_lo = (float)(G.b0 - (double)A.b0);
  A.qmdt = (float)(G.qm * G.dt);
  A.omega_t = (float)omega_at(G.omega, G.t_spin, t);
  return A;
}

}  // namespace

template <int SPEC>
static void launch_tiles(pic_ctx *c, const Args32 &A, int64_t blocks) {
  const TileMaps &M = *reinterpret_cast<const TileMaps *>(c->tile_maps[c->d.tile_shape]);
  if (c->tiles.TI == 8) ++c->launches, k_tiles32<8, 32, SPEC><<<(unsigned)blocks, NT, 0, c->stream>>>(A, c->p32, M);
  else if (c->tiles.TI == 32) ++c->launches, k_tiles32<32, 8, SPEC><<<(unsigned)blocks, NT, 0, c->stream>>>(A, c->p32, M);
  else ++c->launches, k_tiles32<16, 16, SPEC><<<(unsigned)blocks, NT, 0, c->stream>>>(A, c->p32, M);
}

// The six field tensors of every tile shape (at context creation; the arrays
// do not move afterwards).  0 or -1 when the encoder is unavailable or
// rejects a map.
template <int TI, int TJ>
static int encode_maps(pic_ctx *c, void *fn, unsigned char *out) {
  using Enc = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                           const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                           CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  const Grid &G = c->G;
  const cuuint64_t dims[2] = {(cuuint64_t)G.LD, (cuuint64_t)(c->grid_elems / G.LD)};
  const cuuint64_t strides[1] = {(cuuint64_t)G.LD * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)Box<TI, TJ>::WB, (cuuint32_t)Box<TI, TJ>::WI};
  const cuuint32_t estr[2] = {1, 1};
  TileMaps *M = reinterpret_cast<TileMaps *>(out);
  for (int k = 0; k < 6; ++k) {
    const CUresult r = reinterpret_cast<Enc>(fn)(&M->m[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->f32[k], dims, strides,
                                                 box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return -1;
  }
  return 0;
}

int tiles32_setup(pic_ctx *c) {
  static_assert(sizeof(TileMaps) <= sizeof(c->tile_maps[0]), "tensor-map storage");
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return -1;
  // the grid arrays' pitch must be a whole number of 16-byte units
  if ((c->G.LD * sizeof(float)) % 16 != 0 || (c->G.PJ - H - 1 - WOFF) % 4 != 0) return -1;
  if (encode_maps<16, 16>(c, fn, c->tile_maps[0]) || encode_maps<8, 32>(c, fn, c->tile_maps[1]) ||
      encode_maps<32, 8>(c, fn, c->tile_maps[2]))
    return -1;
  // a device copy for the batched ensemble kernel (the arrays never move)
  if (cudaMalloc((void **)&c->d_tile_maps, sizeof c->tile_maps) != cudaSuccess ||
      cudaMemcpy(c->d_tile_maps, c->tile_maps, sizeof c->tile_maps, cudaMemcpyHostToDevice) != cudaSuccess)
    return -1;
  return 0;
}

// the compile-time specialisation of the tile kernel a context takes (the
// monopole one turns each column's node angle by the offset with a short
// series: nth >= 32 keeps that angle below pi / 32)
static int tile_spec(const pic_ctx *c) {
  const pic_desc &d = c->d;
  return c->small_steps && d.r_map == PIC_R_LOG && d.pusher == PIC_VAY
             ? (d.th_map == PIC_TH_LINEAR && d.vacuum == PIC_VAC_MONOPOLE && d.nth >= 32 ? SPEC_MONOPOLE
                : d.th_map == PIC_TH_EQUAL_AREA && d.vacuum == PIC_VAC_MONOPOLE_ROTATOR ? SPEC_ROTATOR
                                                                                         : SPEC_GENERIC)
             : SPEC_GENERIC;
}

int64_t ens_tile_blocks(const pic_ctx *c) {
  if (c->n_used == 0) return 0;
  return c->tiles.nunits + (c->n_used - c->tiles.sorted_end + NT - 1) / NT;
}

void particles32(pic_ctx *c, double t) {
  if (c->n_used == 0) return;
  Args32 A = make_args(c, t);
  const int64_t blocks = ens_tile_blocks(c);
  const int spec = tile_spec(c);
  if (spec == SPEC_MONOPOLE) launch_tiles<SPEC_MONOPOLE>(c, A, blocks);
  else if (spec == SPEC_ROTATOR) launch_tiles<SPEC_ROTATOR>(c, A, blocks);
  else launch_tiles<SPEC_GENERIC>(c, A, blocks);
}

}  // namespace pic

// The bounded device-side wait of the tile kernel, exercised on its own (see
// include/picsar.h): PIC_ETIMEOUT when the wait gave up, PIC_OK when it saw
// its phase complete.
extern "C" int pic_wait_selftest(int64_t polls, int32_t arrive_first, void *stream) {
  if (polls < 1) return pic_fail(PIC_EINVAL, "polls must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  int *d = nullptr;
  PIC_CUDA(cudaMalloc((void **)&d, sizeof(int)));
  int h = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    pic::k_wait_selftest<<<1, 32, 0, st>>>((long long)polls, arrive_first ? 1 : 0, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return pic_cuda_check(e, "wait self-test");
  if (h & pic::ERR_TIMEOUT) return pic_fail(PIC_ETIMEOUT, "the bounded wait gave up (as intended when nothing arrives)");
  return PIC_OK;
}

namespace pic {

size_t ens_tile_arg_bytes() { return sizeof(EnsTileArg); }

// kind = 3 x specialisation + tile shape (0: 16 x 16, 1: 8 x 32, 2: 32 x 8)
int ens_tile_kind(const pic_ctx *c) {
  const int shape = c->tiles.TI == 8 ? 1 : (c->tiles.TI == 32 ? 2 : 0);
  return 3 * tile_spec(c) + shape;
}

void ens_tile_arg(pic_ctx *c, double t, void *out) {
  EnsTileArg a;
  a.A = make_args(c, t);
  a.P = c->p32;
  const int shape = c->tiles.TI == 8 ? 1 : (c->tiles.TI == 32 ? 2 : 0);
  a.maps = reinterpret_cast<const CUtensorMap *>(c->d_tile_maps + (size_t)shape * sizeof(TileMaps));
  memcpy(out, &a, sizeof a);
}

template <int SPEC>
static void ens_tiles_spec(int shape, const EnsTileBatch &B, unsigned blocks, cudaStream_t s) {
  if (shape == 1) k_ens_tiles32<8, 32, SPEC><<<blocks, NT, 0, s>>>(B);
  else if (shape == 2) k_ens_tiles32<32, 8, SPEC><<<blocks, NT, 0, s>>>(B);
  else k_ens_tiles32<16, 16, SPEC><<<blocks, NT, 0, s>>>(B);
}

int ens_tiles32(int kind, const void *args, const int64_t *blocks, int n, cudaStream_t s) {
  const EnsTileArg *T = static_cast<const EnsTileArg *>(args);
  const int spec = kind / 3, shape = kind % 3;
  int launches = 0;
  static thread_local EnsTileBatch B;  // 20 KB: kept off the stack
  for (int first = 0; first < n; first += ENS_TILE_SLOTS) {
    const int m = std::min(ENS_TILE_SLOTS, n - first);
    B.n = m;
    B.off[0] = 0;
    for (int k = 0; k < m; ++k) {
      B.a[k] = T[first + k];
      B.off[k + 1] = B.off[k] + (int)blocks[first + k];
    }
    const unsigned g = (unsigned)B.off[m];
    if (spec == SPEC_MONOPOLE) ens_tiles_spec<SPEC_MONOPOLE>(shape, B, g, s);
    else if (spec == SPEC_ROTATOR) ens_tiles_spec<SPEC_ROTATOR>(shape, B, g, s);
    else ens_tiles_spec<SPEC_GENERIC>(shape, B, g, s);
    ++launches;
  }
  return launches;
}

void ens_flux_from_acc(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s) {
  k_ens_flux<<<(unsigned)blocks, 256, 0, s>>>(tab, L);
}

void flux_from_acc(pic_ctx *c) {
  const Grid &G = c->G;
  dim3 gr((G.nth + 1 + 31) / 32, (G.nr + 2 * G.g + 1 + 7) / 8);
  ++c->launches, k_flux_from_acc<<<gr, dim3(32, 8), 0, c->stream>>>(G.nr, G.nth, G.g, G.PI, G.PJ, G.LD, c->qexp,
                                                     c->acc[0], c->acc[1], c->acc[2], c->F[0], c->F[1], c->F[2]);
}

// Particles per work unit: at least UNIT_MIN, and large enough that a run
// holds no more than about UNIT_TARGET units besides one per tile (two waves of
// 4 CTAs on each of the 152 SMs): a large run keeps one unit per tile, while
// the dense tiles of a small plasma are spread over many CTAs instead of
// holding the whole kernel back on one.
constexpr int64_t UNIT_MIN = 4096, UNIT_TARGET = 2 * 4 * 152;

int64_t sort32(pic_ctx *c) {
  Tiles &T = c->tiles;
  const int64_t n = c->n_used;
  T.nunits = 0;
  if (n == 0) {
    T.sorted_end = 0;
    cudaMemsetAsync(T.start, 0, (T.nbins + 1) * sizeof(int64_t), c->stream);
    return 0;
  }
  // room for the work units first: on failure no particle has moved, every
  // particle takes the unbinned path until a sort succeeds, and the context
  // reports the error
  T.unit = std::max(UNIT_MIN, (n + UNIT_TARGET - 1) / UNIT_TARGET);
  const int64_t ucap = T.ntiles + n / T.unit + 1;
  if (ucap > T.units_cap) {
    cudaStreamSynchronize(c->stream);
    cudaFree(T.units);
    T.units = nullptr;
    T.units_cap = 0;
    T.sorted_end = 0;
    if (cudaMalloc((void **)&T.units, (size_t)ucap * sizeof(long long)) != cudaSuccess) {
      cudaGetLastError();
      c->host_err |= ERR_CAPACITY;
      return -1;
    }
    T.units_cap = ucap;
  }
  Args32 A = make_args(c, 0.0);
  A.mix = c->mix_sort ? 1 : 0;
  c->mix_sort = false;
  int64_t *count = T.cursor;
  cudaMemsetAsync(count, 0, (T.nbins + 1) * sizeof(int64_t), c->stream);
  const unsigned blocks = (unsigned)((n + 255) / 256);
  const int nblk = (int)((T.nbins + SCAN_CHUNK - 1) / SCAN_CHUNK);
  ++c->launches, k_hist<<<blocks, 256, 0, c->stream>>>(A, c->p32, n, count);
  ++c->launches, k_scan_sums<<<nblk, 256, 0, c->stream>>>(count, T.nbins, T.bsum);
  ++c->launches, k_scan_bins<<<1, 1024, 0, c->stream>>>(T.bsum, T.bsum + nblk + 1, nblk);
  ++c->launches, k_scan_apply<<<nblk, 256, 0, c->stream>>>(count, T.start, T.nbins, T.bsum + nblk + 1, nblk);
  ++c->launches, k_scatter_cells<<<blocks, 256, 0, c->stream>>>(A, c->p32, c->q32, n, count);
  // the work units of the tile kernel (n bounds the live count from above)
  const unsigned tb = (unsigned)((T.ntiles + 255) / 256);
  const int ublk = (int)((T.ntiles + SCAN_CHUNK - 1) / SCAN_CHUNK);
  ++c->launches, k_unit_count<<<tb, 256, 0, c->stream>>>(T.start, T.tc, T.ntiles, T.unit, T.ucount);
  ++c->launches, k_scan_sums<<<ublk, 256, 0, c->stream>>>(T.ucount, T.ntiles, T.usum);
  ++c->launches, k_scan_bins<<<1, 1024, 0, c->stream>>>(T.usum, T.usum + ublk + 1, ublk);
  ++c->launches, k_scan_apply<<<ublk, 256, 0, c->stream>>>(T.ucount, T.ucount, T.ntiles, T.usum + ublk + 1, ublk);
  ++c->launches, k_unit_fill<<<tb, 256, 0, c->stream>>>(T.ucount, T.ntiles, T.units);
  // particles in cell bins: everything before the bin of removed ones; units
  cudaMemcpyAsync(c->h_pinned, T.start + (int64_t)T.ntiles * T.tc, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(c->h_pinned + 1, T.ucount + T.ntiles, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  const int64_t live = c->h_pinned[0];
  T.nunits = c->h_pinned[1];
  Parts32 tmp = c->p32;
  c->p32 = c->q32;
  c->q32 = tmp;
  c->n_used = live;
  T.sorted_end = live;
  return live;
}

void ens_sort_scratch_free(EnsSortScratch &sc) {
  if (sc.h) cudaFreeHost(sc.h);
  if (sc.d) cudaFree(sc.d);
  sc = EnsSortScratch{};
}

int ens_sort32(pic_ctx *const *cs, int m, cudaStream_t st, EnsSortScratch &sc, int64_t *kernels) {
  *kernels = 0;
  std::vector<pic_ctx *> due;
  for (int k = 0; k < m; ++k) {
    pic_ctx *c = cs[k];
    if (c->n_used == 0) {  // nothing to order: as sort32
      sort32(c);
      c->steps_since_sort = 0;
      continue;
    }
    due.push_back(c);
  }
  const int nd = (int)due.size();
  if (nd == 0) return PIC_OK;
  // room for each member's work units (reallocated after the device is idle
  // on the stream: a previous graph may still read the old list)
  bool synced = false;
  for (pic_ctx *c : due) {
    Tiles &T = c->tiles;
    T.unit = std::max(UNIT_MIN, (c->n_used + UNIT_TARGET - 1) / UNIT_TARGET);
    const int64_t ucap = T.ntiles + c->n_used / T.unit + 1;
    if (ucap <= T.units_cap) continue;
    if (!synced) { PIC_CUDA(cudaStreamSynchronize(st)); synced = true; }
    cudaFree(T.units);
    T.units = nullptr;
    T.units_cap = 0;
    T.sorted_end = 0;
    T.nunits = 0;
    PIC_CUDA(cudaMalloc((void **)&T.units, (size_t)ucap * sizeof(long long)));
    T.units_cap = ucap;
  }
  // phase maps: {member, block} per block of each launch
  enum { M_ZERO, M_PART, M_BINS, M_TOP, M_TILE, M_UBINS, M_UTOP, M_N };
  std::vector<int2> mp[M_N];
  auto add = [&](int q, int k, int64_t blocks) {
    for (int64_t b = 0; b < blocks; ++b) mp[q].push_back(make_int2(k, (int)b));
  };
  std::vector<EnsSortArg> tab(nd);
  const size_t tab_bytes = (size_t)nd * sizeof(EnsSortArg);
  for (int k = 0; k < nd; ++k) {
    pic_ctx *c = due[k];
    Tiles &T = c->tiles;
    EnsSortArg &E = tab[k];
    E.A = make_args(c, 0.0);
    E.A.mix = c->mix_sort ? 1 : 0;
    c->mix_sort = false;
    E.S = c->p32;
    E.D = c->q32;
    E.n = c->n_used;
    E.count = T.cursor;
    E.start = T.start;
    E.bsum = T.bsum;
    E.nbins = T.nbins;
    E.nblk = (int)((T.nbins + SCAN_CHUNK - 1) / SCAN_CHUNK);
    E.ublk = (int)((T.ntiles + SCAN_CHUNK - 1) / SCAN_CHUNK);
    E.ntiles = T.ntiles;
    E.tc = T.tc;
    E.ucount = T.ucount;
    E.usum = T.usum;
    E.units = T.units;
    E.unit = T.unit;
    E.err = c->d_err;
    add(M_ZERO, k, (T.nbins + 1 + 255) / 256);
    add(M_PART, k, (E.n + 255) / 256);
    add(M_BINS, k, E.nblk);
    add(M_TOP, k, 1);
    add(M_TILE, k, (T.ntiles + 255) / 256);
    add(M_UBINS, k, E.ublk);
    add(M_UTOP, k, 1);
  }
  // one buffer: the table, the maps and the read-back values
  size_t at[M_N + 1];
  at[0] = (tab_bytes + 255) / 256 * 256;
  for (int q = 0; q < M_N; ++q) at[q + 1] = at[q] + (mp[q].size() * sizeof(int2) + 255) / 256 * 256;
  const size_t out_at = at[M_N], bytes = out_at + (size_t)nd * 3 * sizeof(int64_t);
  if (bytes > sc.cap) {
    PIC_CUDA(cudaStreamSynchronize(st));
    ens_sort_scratch_free(sc);
    PIC_CUDA(cudaMallocHost((void **)&sc.h, bytes));
    PIC_CUDA(cudaMalloc((void **)&sc.d, bytes));
    sc.cap = bytes;
  }
  for (int k = 0; k < nd; ++k) tab[k].out = reinterpret_cast<int64_t *>(sc.d + out_at) + 3 * k;
  memcpy(sc.h, tab.data(), tab_bytes);
  for (int q = 0; q < M_N; ++q) memcpy(sc.h + at[q], mp[q].data(), mp[q].size() * sizeof(int2));
  PIC_CUDA(cudaMemcpyAsync(sc.d, sc.h, out_at, cudaMemcpyHostToDevice, st));
  const EnsSortArg *dt = reinterpret_cast<const EnsSortArg *>(sc.d);
  auto L = [&](int q) {
    EnsList x;
    x.blk = reinterpret_cast<const int2 *>(sc.d + at[q]);
    return x;
  };
  auto nb = [&](int q) { return (unsigned)mp[q].size(); };
  k_ens_sort_zero<<<nb(M_ZERO), 256, 0, st>>>(dt, L(M_ZERO));
  k_ens_hist<<<nb(M_PART), 256, 0, st>>>(dt, L(M_PART));
  k_ens_scan_sums<<<nb(M_BINS), 256, 0, st>>>(dt, L(M_BINS), 0);
  k_ens_scan_bins<<<nb(M_TOP), 1024, 0, st>>>(dt, L(M_TOP), 0);
  k_ens_scan_apply<<<nb(M_BINS), 256, 0, st>>>(dt, L(M_BINS), 0);
  k_ens_scatter<<<nb(M_PART), 256, 0, st>>>(dt, L(M_PART));
  k_ens_unit_count<<<nb(M_TILE), 256, 0, st>>>(dt, L(M_TILE));
  k_ens_scan_sums<<<nb(M_UBINS), 256, 0, st>>>(dt, L(M_UBINS), 1);
  k_ens_scan_bins<<<nb(M_UTOP), 1024, 0, st>>>(dt, L(M_UTOP), 1);
  k_ens_scan_apply<<<nb(M_UBINS), 256, 0, st>>>(dt, L(M_UBINS), 1);
  k_ens_unit_fill<<<nb(M_TILE), 256, 0, st>>>(dt, L(M_TILE));
  k_ens_sort_out<<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(dt, nd);
  PIC_CUDA(cudaGetLastError());
  PIC_CUDA(cudaMemcpyAsync(sc.h + out_at, sc.d + out_at, (size_t)nd * 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  PIC_CUDA(cudaStreamSynchronize(st));
  *kernels = 12;
  const int64_t *out = reinterpret_cast<const int64_t *>(sc.h + out_at);
  for (int k = 0; k < nd; ++k) {
    pic_ctx *c = due[k];
    Tiles &T = c->tiles;
    std::swap(c->p32, c->q32);
    c->n_used = out[3 * k];
    T.sorted_end = out[3 * k];
    T.nunits = out[3 * k + 1];
    c->host_err |= (int)out[3 * k + 2];
    c->steps_since_sort = 0;
    c->launches += 10;  // the kernels of its own sort (sort32)
  }
  return PIC_OK;
}

void charge32(pic_ctx *c, double *Q, double *Qa) {
  if (c->n_used == 0) return;
  // particles keep whole-grid rows: a radial slab's arrays start at row i0
  ++c->launches, k_charge32<<<(unsigned)((c->n_used + 255) / 256), 256, 0, c->stream>>>(c->G.PI - c->G.i0, c->G.PJ, c->G.LD, c->p32,
                                                                        c->n_used, Q, Qa);
}

void reduce_particles32(pic_ctx *c) {
  if (c->n_used == 0) return;
  // a fixed grid (4 blocks per SM) keeps the same-address atomics few
  ++c->launches, k_reduce32<<<4 * 152, 256, 0, c->stream>>>(c->p32, c->n_used, c->G.qm, c->d_acc,
                                                                        c->d_cnt + CNT_LIVE);
}

}  // namespace pic

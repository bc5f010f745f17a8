// fields.cu -- grid-sized kernels beside the particle hot path (FP64):
//   Yee leapfrog in integral form (App. A, Eqs. discreteeq, erpolarupdate) with
//   conducting radial boundaries (Sec. 3.4.1), the lossy layer (Eq. EBcond),
//   the 1-2-1 current filter with the polar remap (App. B), axis ghost
//   columns and FP32 gather copies, surface pair injection (Sec. 5.3,
//   Eq. volinjeq) and the Gauss-law / energy diagnostics.
// All metric factors are precomputed per row and per column (pic::Metric), so
// the kernels are pure streaming stencils over the padded arrays.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "pic_internal.h"

namespace pic {

namespace {

constexpr int BX = 32, BY = 8;

inline dim3 grid2(int ni, int nj) { return dim3((nj + BX - 1) / BX, (ni + BY - 1) / BY); }

// B <- B - h c curl E over the faces of the primary grid (first three lines of
// Eq. discreteeq).  One thread per node (i, j), 0 <= i <= nr, 0 <= j <= nth.
// (the factors of dt / 2 and the metric are folded into the row and column
// coefficient tables of Metric: a few FP64 FMAs per node, the rate that
// limits this kernel)
__device__ __forceinline__ void b_half_node(const Grid &G, int i, int j, const double *__restrict__ Er,
                                            const double *__restrict__ Et, const double *__restrict__ Ep,
                                            double *__restrict__ Br, double *__restrict__ Bt,
                                            double *__restrict__ Bp) {
  if (i > G.nr || j > G.nth) return;
  const Metric &m = G.m;
  const int ri = i + G.PI, cj = j + G.PJ;
  const size_t o = gidx(G, i, j);
  if (j < G.nth)  // B_r at (i, j+1/2)
    Br[o] += m.bR[ri] * (Ep[o] * m.cB1[cj] - Ep[o + 1] * m.cB2[cj]);
  if (i < G.nr) {
    const double t0 = m.bT0[ri], t1 = m.bT1[ri];
    if (j >= 1 && j < G.nth)  // B_th at (i+1/2, j); zero on the axis
      Bt[o] += t1 * Ep[o + G.LD] - t0 * Ep[o];
    if (j < G.nth)  // B_ph at (i+1/2, j+1/2)
      Bp[o] += (t0 * Et[o] - t1 * Et[o + G.LD]) - (Er[o] - Er[o + 1]) * (m.bP[ri] * m.inv_dth_t[cj]);
  }
}

__global__ void k_b_half(Grid G, const double *__restrict__ Er, const double *__restrict__ Et,
                         const double *__restrict__ Ep, double *__restrict__ Br, double *__restrict__ Bt,
                         double *__restrict__ Bp) {
  b_half_node(G, blockIdx.y * BY + threadIdx.y, blockIdx.x * BX + threadIdx.x, Er, Et, Ep, Br, Bt, Bp);
}

// E <- E + dt c curl B - F / dA over the faces of the dual grid (last three
// lines of Eq. discreteeq; E_r on the axis by Eq. erpolarupdate, obtained here
// from the same formula with sin(tb_{-1}) = sin(tb_{nth}) = 0 and the cap
// areas in inv_dcos_tb).  E_th, E_ph stay 0 on the conductors (i = 0, nr) and
// E_ph on the axis.
__device__ __forceinline__ void e_full_node(const Grid &G, int i, int j, double *__restrict__ Er,
                                            double *__restrict__ Et, double *__restrict__ Ep,
                                            const double *__restrict__ Br, const double *__restrict__ Bt,
                                            const double *__restrict__ Bp, const double *__restrict__ Fr,
                                            const double *__restrict__ Ft, const double *__restrict__ Fp) {
  if (i > G.nr || j > G.nth) return;
  const Metric &m = G.m;
  const int ri = i + G.PI, cj = j + G.PJ;
  const size_t o = gidx(G, i, j);
  if (i < G.nr)  // E_r at (i+1/2, j)
    Er[o] += m.eR[ri] * (Bp[o] * m.cE1[cj] - Bp[o - 1] * m.cE2[cj]) - Fr[o] * (m.inv_area_h[ri] * m.inv_dcos_tb[cj]);
  // E_th, E_ph stay 0 on a conductor; a slab's open side is an interior row
  if ((i >= 1 || G.open_lo) && (i < G.nr || G.open_hi)) {
    const double t0 = m.eT0[ri], t1 = m.eT1[ri], id2 = m.inv_dr2_h[ri];
    if (j < G.nth)  // E_th at (i, j+1/2)
      Et[o] += (t0 * Bp[o - G.LD] - t1 * Bp[o]) - Ft[o] * (m.cF[cj] * id2);
    if (j >= 1 && j < G.nth) {  // E_ph at (i, j)
      const double idt = m.inv_dtb[cj];
      Ep[o] += ((t1 * Bt[o] - t0 * Bt[o - G.LD]) - (Br[o] - Br[o - 1]) * (m.eP[ri] * idt)) - Fp[o] * (idt * id2);
    }
  }
}

__global__ void k_e_full(Grid G, double *__restrict__ Er, double *__restrict__ Et, double *__restrict__ Ep,
                         const double *__restrict__ Br, const double *__restrict__ Bt,
                         const double *__restrict__ Bp, const double *__restrict__ Fr,
                         const double *__restrict__ Ft, const double *__restrict__ Fp) {
  e_full_node(G, blockIdx.y * BY + threadIdx.y, blockIdx.x * BX + threadIdx.x, Er, Et, Ep, Br, Bt, Bp, Fr, Ft, Fp);
}

// Lossy layer, Eq. (EBcond): every component times 1 - sigma* at its own
// radial stagger, rows i0..nr.
__device__ __forceinline__ void lossy_node(const Grid &G, int i, int j, double *Er, double *Et, double *Ep,
                                           double *Br, double *Bt, double *Bp) {
  if (i > G.nr || j > G.nth) return;
  const size_t o = gidx(G, i, j);
  const double kn = G.m.keep_n[i + G.PI], kh = G.m.keep_h[i + G.PI];
  Er[o] *= kh; Bt[o] *= kh; Bp[o] *= kh;
  Et[o] *= kn; Ep[o] *= kn; Br[o] *= kn;
}

__global__ void k_lossy(Grid G, double *Er, double *Et, double *Ep, double *Br, double *Bt, double *Bp, int i0) {
  lossy_node(G, i0 + blockIdx.y * BY + threadIdx.y, blockIdx.x * BX + threadIdx.x, Er, Et, Ep, Br, Bt, Bp);
}

// Axisymmetric continuation of the half-integer-j components into columns -1
// and nth (B_r even; E_th, B_ph odd).
__device__ __forceinline__ void ghost_row(const Grid &G, int i, double *Et, double *Br, double *Bp) {
  if (i > G.nr) return;
  const size_t n0 = gidx(G, i, -1), s0 = gidx(G, i, G.nth);
  Et[n0] = -Et[n0 + 1]; Br[n0] = Br[n0 + 1]; Bp[n0] = -Bp[n0 + 1];
  Et[s0] = -Et[s0 - 1]; Br[s0] = Br[s0 - 1]; Bp[s0] = -Bp[s0 - 1];
}

__global__ void k_axis_ghosts(Grid G, double *Et, double *Br, double *Bp) {
  ghost_row(G, blockIdx.x * blockDim.x + threadIdx.x, Et, Br, Bp);
}

// FP32 gather copies of the six components (the gather-prep step of the FP32
// path) over rows -g..nr+g and columns -1..nth: every node the gather can
// read.  The FP64 fields are zero outside rows 0..nr and columns -1..nth (no
// kernel writes there), and so are the FP32 copies from their allocation, so
// the padding beyond needs no copy.
__device__ __forceinline__ void copy32_node(const Grid &G, int i, int j, const double *__restrict__ a0,
                                            const double *__restrict__ a1, const double *__restrict__ a2,
                                            const double *__restrict__ a3, const double *__restrict__ a4,
                                            const double *__restrict__ a5, float *b0, float *b1, float *b2,
                                            float *b3, float *b4, float *b5) {
  if (i > G.nr + G.g || j > G.nth) return;
  const size_t k = gidx(G, i, j);
  b0[k] = (float)a0[k]; b1[k] = (float)a1[k]; b2[k] = (float)a2[k];
  b3[k] = (float)a3[k]; b4[k] = (float)a4[k]; b5[k] = (float)a5[k];
}

__global__ void k_copy32(Grid G, const double *__restrict__ a0, const double *__restrict__ a1,
                         const double *__restrict__ a2, const double *__restrict__ a3,
                         const double *__restrict__ a4, const double *__restrict__ a5, float *b0, float *b1,
                         float *b2, float *b3, float *b4, float *b5) {
  copy32_node(G, -G.g + (int)(blockIdx.y * BY + threadIdx.y), (int)(blockIdx.x * BX + threadIdx.x) - 1, a0, a1, a2,
              a3, a4, a5, b0, b1, b2, b3, b4, b5);
}

// One 1-2-1 pass (Eq. filtereq) with the polar remap of App. B: weights V_l(j)
// fold the part that would leave through the axis back onto the mirror point,
// + for integer-j arrays (F_r, F_ph, charge) and - for the half-integer-j F_th.
// Rows outside the ghost band -g..nr+g are not kept.
__device__ __forceinline__ void filter_node(const Grid &G, int i, int j, const double *__restrict__ in,
                                            double *__restrict__ out, int half_j) {
  const int nj = half_j ? G.nth : G.nth + 1;
  if (i > G.nr + G.g || j >= nj) return;
  double vm, v0 = 0.5, vp;
  if (half_j) {
    vm = j == 0 ? 0.0 : 0.25;
    vp = j == G.nth - 1 ? 0.0 : 0.25;
    if (j == 0) v0 -= 0.25;
    if (j == G.nth - 1) v0 -= 0.25;
  } else {
    vm = j == 0 ? 0.0 : (j == 1 ? 0.5 : 0.25);
    vp = j == G.nth ? 0.0 : (j == G.nth - 1 ? 0.5 : 0.25);
  }
  const size_t o = gidx(G, i, j);
  double s = 0.0;
#pragma unroll
  for (int k = -1; k <= 1; ++k) {
    const int ii = i + k;
    if (ii < -G.g || ii > G.nr + G.g) continue;
    const size_t q = o + (ptrdiff_t)k * G.LD;
    double row = vm * in[q - 1] + v0 * in[q] + vp * in[q + 1];
    s += (k == 0 ? 0.5 : 0.25) * row;
  }
  out[o] = s;
}

__global__ void k_filter(Grid G, const double *__restrict__ in, double *__restrict__ out, int half_j) {
  filter_node(G, -G.g + (int)(blockIdx.y * BY + threadIdx.y), blockIdx.x * BX + threadIdx.x, in, out, half_j);
}

// Surface charge per meridional cell: the jump of E_r across the conductor,
// total E_r at (1/2, j) minus the analytic inside field's E_r at (r0, theta_j)
// (zero for the monopole fields), averaged over the cell's two nodes.
__device__ __forceinline__ void sigma_cell(const Grid &G, int j, const double *__restrict__ Er, double t, double *sig,
                                           long long *smax) {
  if (j >= G.nth) return;
  const Metric &m = G.m;
  const double rb0 = m.r_h[G.PI];
  double E[3], B[3], Ei[3];
  const Vac<double> V{G.vacuum, G.b0, G.r_min, omega_at(G.omega, G.t_spin, t)};
  double e[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const double st = m.sin_t[j + h + G.PJ], ct = m.cos_t[j + h + G.PJ];
    vacuum_field<double>(V, rb0, st, ct, false, E, B);
    vacuum_field<double>(V, G.r_min, st, ct, true, Ei, B);
    e[h] = (Er[gidx(G, 0, j + h)] + E[0]) - Ei[0];
  }
  const double s = 0.5 * (e[0] + e[1]);
  sig[j] = s;
  if (smax) atomicMax(smax, __double_as_longlong(fabs(s)));
}

__global__ void k_inject_sigma(Grid G, const double *__restrict__ Er, double t, double *sig, long long *smax) {
  sigma_cell(G, blockIdx.x * blockDim.x + threadIdx.x, Er, t, sig, smax);
}

// One 1-2-1 pass over sigma along theta; each polar cell is its own mirror
// image across the axis.
__device__ __forceinline__ void smooth_cell(int j, int nth, const double *__restrict__ in, double *out,
                                            long long *smax) {
  if (j >= nth) return;
  const double a = in[j > 0 ? j - 1 : 0], c = in[j < nth - 1 ? j + 1 : nth - 1];
  const double s = ((a + 2.0 * in[j]) + c) * 0.25;
  out[j] = s;
  if (smax) atomicMax(smax, __double_as_longlong(fabs(s)));
}

__global__ void k_inject_smooth(int nth, const double *__restrict__ in, double *out, long long *smax) {
  smooth_cell(blockIdx.x * blockDim.x + threadIdx.x, nth, in, out, smax);
}

// SplitMix64 (Steele, Lea and Flood 2014) as a counter-based generator:
// output n + 1 of the stream seeded with `seed` is the variant-13 mix of
// seed + (n + 1) times the golden-ratio increment.
__device__ inline uint64_t splitmix64_out(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct InjectRule {
  int mode, npp;
  double finj, q;       // q: VARIABLE, |charge| per particle
  uint64_t seed, step;  // VARIABLE: generator key (seed, step * nth + j)
};

// Pairs injected into cell j and the |charge| of each (Eq. volinjeq).
__device__ inline int inject_count(const Grid &G, const InjectRule &R, int j, double sg, double sm, double dA,
                                   double &w, bool &capped) {
  capped = false;
  if (R.mode == PIC_INJECT_VARIABLE) {
    const double x = R.finj * fabs(sg) * dA / R.q;
    w = R.q;
    if (!(fabs(sg) > 1e-12 * sm && x > 0.0)) return 0;
    int m;
    if (x >= R.npp + 1.0) {
      m = R.npp + 1;
    } else {
      const double fl = floor(x);
      const double u = (double)(splitmix64_out(R.seed, R.step * (uint64_t)G.nth + (uint64_t)j) >> 11) *
                       (1.0 / 9007199254740992.0);
      m = (int)fl + (u < x - fl ? 1 : 0);
    }
    if (m > R.npp) { m = R.npp; capped = true; }
    return m;
  }
  w = R.finj * fabs(sg) * dA / R.npp;
  return (fabs(sg) > 1e-12 * sm && w > 0.0) ? R.npp : 0;
}

// One thread per slot (j, k, sign) of the 2 npp nth reserved this step; slots
// past a cell's count keep zero charge (free).
// (every lane of a warp calls it: the exponent is raised warp-wide)
template <bool FP32>
__device__ __forceinline__ void inject_slot(int64_t idx, const Grid &G, const double *__restrict__ sig,
                                            const long long *smax, const Parts64 &P, const Parts32 &Q, int64_t base,
                                            int64_t id0, const InjectRule &R, long long *cnt, long long *capped_cnt,
                                            long long *qexp) {
  const int npp = R.npp;
  int qe = (int)QEXP_NONE;
  if (idx < (int64_t)G.nth * npp * 2) {
    const int j = (int)(idx / (2 * npp)), k = (int)((idx / 2) % npp), s = (int)(idx % 2);
    const double sm = __longlong_as_double(*smax), sg = sig[j];
    const double r0 = G.r_min;
    const double dA = 2.0 * PI_D * r0 * r0 * (G.m.cos_t[j + G.PJ] - G.m.cos_t[j + 1 + G.PJ]);
    double w;
    bool capped;
    const int m = inject_count(G, R, j, sg, sm, dA, w, capped);
    if (capped && k == 0 && s == 0) add_ll(capped_cnt, 1LL);
    const bool on = k < m;
    const int64_t slot = base + idx;
    const double qv = on ? (s == 0 ? w : -w) : 0.0;
    const double oy = (k + 0.5) / (on ? m : npp);
    if (FP32) {
      Q.cell[slot] = ((uint32_t)(0 + CELL_BIAS) << 16) | (uint32_t)j;
      Q.dx[slot] = 0.5f;
      Q.dy[slot] = (float)oy;
      Q.ur[slot] = Q.ut[slot] = Q.up[slot] = 0.0f;
      Q.qw[slot] = (float)qv;
      Q.id[slot] = id0 + idx;
      if (on) qe = charge_exp(fabsf((float)qv));
    } else {
      P.x1[slot] = 0.5;
      P.x2[slot] = j + oy;
      P.ur[slot] = P.ut[slot] = P.up[slot] = 0.0;
      P.qw[slot] = qv;
      P.id[slot] = id0 + idx;
    }
    if (on) add_ll(cnt, 1LL);
  }
  if (FP32) raise_qexp(qexp, qe);  // every lane of the warp reaches this
}

template <bool FP32>
__global__ void k_inject_write(Grid G, const double *__restrict__ sig, const long long *smax, Parts64 P,
                               Parts32 Q, int64_t base, int64_t id0, InjectRule R, long long *cnt,
                               long long *capped_cnt, long long *qexp) {
  inject_slot<FP32>(blockIdx.x * (int64_t)blockDim.x + threadIdx.x, G, sig, smax, P, Q, base, id0, R, cnt,
                    capped_cnt, qexp);
}

__device__ inline double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Integral Gauss law per dual cell: G = flux of E out of the dual cell of node
// (i, j) (caps close at the axis); d = G - Qbar.  snapshot: store d; else
// reduce max |d - d_0| and max |Q| over interior nodes 1 <= i <= imax.
__global__ void k_gauss(Grid G, const double *__restrict__ Er, const double *__restrict__ Et,
                        const double *__restrict__ Qf, const double *__restrict__ Qa, double *snap, int ilo, int imax,
                        int snapshot, long long *gmax, long long *qmax) {
  const int j = blockIdx.x * BX + threadIdx.x, i = ilo + blockIdx.y * BY + threadIdx.y;
  double v = 0.0, qa = 0.0;
  if (i <= imax && j <= G.nth) {
    const Metric &m = G.m;
    const int ri = i + G.PI, cj = j + G.PJ;
    const size_t o = gidx(G, i, j);
    const double dc = 1.0 / m.inv_dcos_tb[cj];
    const double ar = 2.0 * PI_D * m.r_h[ri] * m.r_h[ri], al = 2.0 * PI_D * m.r_h[ri - 1] * m.r_h[ri - 1];
    const double side = PI_D * (m.r_h[ri] * m.r_h[ri] - m.r_h[ri - 1] * m.r_h[ri - 1]);
    double g = Er[o] * ar * dc - Er[o - G.LD] * al * dc + (Et[o] * m.sin_tb[cj] - Et[o - 1] * m.sin_tb[cj - 1]) * side;
    double d = g - Qf[o];
    if (snapshot) snap[o] = d;
    else v = fabs(d - snap[o]);
    qa = Qa[o];
  }
  v = warp_max(v);
  qa = warp_max(qa);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(gmax, __double_as_longlong(v));
    atomicMax(qmax, __double_as_longlong(qa));
  }
}

// rows 0..imax (a slab leaves its open outer interface row to the neighbour)
__global__ void k_field_energy(Grid G, const double *f0, const double *f1, const double *f2, const double *f3,
                               const double *f4, const double *f5, int imax, double *acc) {
  const int j = blockIdx.x * BX + threadIdx.x, i = blockIdx.y * BY + threadIdx.y;
  double e = 0.0;
  if (i <= imax && j <= G.nth) {
    const Metric &m = G.m;
    const int ri = i + G.PI, cj = j + G.PJ;
    const size_t o = gidx(G, i, j);
    const double *fs[6] = {f0, f1, f2, f3, f4, f5};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const int si = stag_i(c), sj = stag_j(c);
      if ((si && i >= G.nr) || (sj && j >= G.nth)) continue;
      const double vr = si ? m.vol_r_h[ri] : m.vol_r_n[ri];
      const double vt = sj ? m.vol_t_h[cj] : m.vol_t_n[cj];
      const double v = fs[c][o];
      e += 0.5 * v * v * vr * vt;
    }
  }
  e = warp_sum(e);
  if ((threadIdx.x & 31) == 0) atomicAdd(acc, e);
}

// ---- the same kernels over the members of an ensemble ----------------------
// 256-thread blocks; a member's 2-D node blocks (32 x 8, as the kernels above
// take them) are numbered row-major across its grid.
struct Node2 {
  int i, j;
};
__device__ inline Node2 node_of(unsigned b, int nj, int i_first) {
  const unsigned gx = (unsigned)(nj + BX - 1) / BX;
  return Node2{i_first + (int)((b / gx) * BY + (threadIdx.x >> 5)), (int)((b % gx) * BX + (threadIdx.x & 31))};
}

// pass `pass` of the filter on all three flux components: even passes read
// the deposit's buffers and write the scratch, odd passes the reverse
__global__ void k_ens_filter(const EnsFieldArg *__restrict__ tab, EnsList L, int pass) {
  const int2 e = L.blk[blockIdx.x];
  const EnsFieldArg &E = tab[e.x];
  const Grid &G = E.G;
  const unsigned per = (unsigned)((G.nth + 1 + BX - 1) / BX) * (unsigned)((G.nr + 2 * G.g + 1 + BY - 1) / BY);
  const unsigned b = (unsigned)e.y;
  const int comp = (int)(b / per);
  const Node2 n = node_of(b % per, G.nth + 1, -G.g);
  const double *in = (pass & 1) ? E.Ftmp[comp] : E.Fin[comp];
  double *out = (pass & 1) ? E.Fin[comp] : E.Ftmp[comp];
  filter_node(G, n.i, n.j, in, out, comp == 1);
}

__global__ void k_ens_b_half(const EnsFieldArg *__restrict__ tab, EnsList L) {
  const int2 e = L.blk[blockIdx.x];
  const EnsFieldArg &E = tab[e.x];
  const Node2 n = node_of((unsigned)e.y, E.G.nth + 1, 0);
  b_half_node(E.G, n.i, n.j, E.f[ER], E.f[ETH], E.f[EPH], E.f[BR], E.f[BTH], E.f[BPH]);
}

__global__ void k_ens_e_full(const EnsFieldArg *__restrict__ tab, EnsList L) {
  const int2 e = L.blk[blockIdx.x];
  const EnsFieldArg &E = tab[e.x];
  const Node2 n = node_of((unsigned)e.y, E.G.nth + 1, 0);
  e_full_node(E.G, n.i, n.j, E.f[ER], E.f[ETH], E.f[EPH], E.f[BR], E.f[BTH], E.f[BPH], E.Fout[0], E.Fout[1],
              E.Fout[2]);
}

__global__ void k_ens_lossy(const EnsFieldArg *__restrict__ tab, EnsList L) {
  const int2 e = L.blk[blockIdx.x];
  const EnsFieldArg &E = tab[e.x];
  const Node2 n = node_of((unsigned)e.y, E.G.nth + 1, E.lossy_i0);
  lossy_node(E.G, n.i, n.j, E.f[0], E.f[1], E.f[2], E.f[3], E.f[4], E.f[5]);
}

// axis ghosts; block 0 of a member that injects also clears the surface
// charge maximum its injection will raise later in the step
__global__ void k_ens_ghosts(const EnsFieldArg *__restrict__ tab, EnsList L) {
  const int2 e = L.blk[blockIdx.x];
  const EnsFieldArg &E = tab[e.x];
  const unsigned b = (unsigned)e.y;
  if (b == 0 && threadIdx.x == 0 && E.inject) E.cnt[CNT_SMAX] = 0;
  ghost_row(E.G, (int)(b * blockDim.x + threadIdx.x), E.f[ETH], E.f[BR], E.f[BPH]);
}

__global__ void k_ens_copy32(const EnsFieldArg *__restrict__ tab, EnsList L) {
  const int2 e = L.blk[blockIdx.x];
  const EnsFieldArg &E = tab[e.x];
  const Node2 n = node_of((unsigned)e.y, E.G.nth + 2, -E.G.g);
  copy32_node(E.G, n.i, n.j - 1, E.f[0], E.f[1], E.f[2], E.f[3], E.f[4], E.f[5], E.f32[0], E.f32[1], E.f32[2],
              E.f32[3], E.f32[4], E.f32[5]);
}

__device__ inline InjectRule ens_rule(const EnsFieldArg &E) {
  return InjectRule{E.inject, E.npp, E.f_inj, E.inject_q, E.inject_seed, E.inj_step};
}

__global__ void k_ens_sigma(const EnsFieldArg *__restrict__ tab, EnsList L) {
  const int2 e = L.blk[blockIdx.x];
  const EnsFieldArg &E = tab[e.x];
  const int j = (int)(((unsigned)e.y) * blockDim.x + threadIdx.x);
  sigma_cell(E.G, j, E.f[ER], E.t_inj, E.sig, E.inject_smooth ? nullptr : E.cnt + CNT_SMAX);
}

__global__ void k_ens_smooth(const EnsFieldArg *__restrict__ tab, EnsList L, int pass) {
  const int2 e = L.blk[blockIdx.x];
  const EnsFieldArg &E = tab[e.x];
  const int j = (int)(((unsigned)e.y) * blockDim.x + threadIdx.x), nth = E.G.nth;
  const double *in = (pass & 1) ? E.sig + (nth + 1) : E.sig;
  double *out = (pass & 1) ? E.sig : E.sig + (nth + 1);
  smooth_cell(j, nth, in, out, pass == E.inject_smooth - 1 ? E.cnt + CNT_SMAX : nullptr);
}

__global__ void k_ens_write(const EnsFieldArg *__restrict__ tab, EnsList L) {
  const int2 e = L.blk[blockIdx.x];
  const EnsFieldArg &E = tab[e.x];
  const int64_t idx = (int64_t)((unsigned)e.y) * blockDim.x + threadIdx.x;
  const double *sig = (E.inject_smooth & 1) ? E.sig + (E.G.nth + 1) : E.sig;
  const Parts64 none;
  inject_slot<true>(idx, E.G, sig, E.cnt + CNT_SMAX, none, E.p32, E.inj_base, E.inj_id0, ens_rule(E),
                    E.cnt + CNT_INJECTED, E.cnt + CNT_CAPPED, E.qexp);
}

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace

int ens_blocks(const pic_ctx *c, int kind) {
  const Grid &G = c->G;
  const int gx = div_up(G.nth + 1, BX);
  switch (kind) {
    case ENS_FLUX: return gx * div_up(G.nr + 2 * G.g + 1, BY);
    case ENS_FILTER: return c->d.n_filt > 0 ? 3 * gx * div_up(G.nr + 2 * G.g + 1, BY) : 0;
    case ENS_NODES: return gx * div_up(G.nr + 1, BY);
    case ENS_LOSSY: {
      if (c->d.absorb_profile == PIC_ABSORB_NONE || c->d.absorb_cells <= 0) return 0;
      const int i0 = std::max(0, G.nr - G.absorb_cells - 1);
      return gx * div_up(G.nr + 1 - i0, BY);
    }
    case ENS_GHOSTS: return div_up(G.nr + 1, 256);
    case ENS_COPY32: return div_up(G.nth + 2, BX) * div_up(G.nr + 2 * G.g + 1, BY);
    case ENS_SIGMA: return c->d.inject ? div_up(G.nth, 256) : 0;
    case ENS_WRITE: return c->d.inject ? div_up((int64_t)G.nth * c->d.pairs_per_cell * 2, 256) : 0;
    default: return 0;
  }
}

void ens_fill_field_arg(const pic_ctx *c, EnsFieldArg *a) {
  memset(a, 0, sizeof *a);
  a->G = c->G;
  for (int k = 0; k < 6; ++k) { a->f[k] = c->f[k]; a->f32[k] = c->f32[k]; }
  for (int k = 0; k < 3; ++k) {
    a->Fin[k] = c->F[k];
    a->Ftmp[k] = c->Ft[k];
    a->Fout[k] = (c->d.n_filt & 1) ? c->Ft[k] : c->F[k];
    a->acc[k] = c->acc[k];
  }
  a->grid_elems = c->grid_elems;
  a->cnt = c->d_cnt;
  a->qexp = c->qexp;
  a->sig = c->sig;
  a->p32 = c->p32;
  a->f_inj = c->d.f_inj;
  a->inject_q = c->d.inject_q;
  a->inject_seed = c->d.inject_seed;
  a->inject = c->d.inject;
  a->npp = c->d.pairs_per_cell;
  a->inject_smooth = c->d.inject_smooth;
  a->n_filt = c->d.n_filt;
  a->lossy_i0 = (c->d.absorb_profile != PIC_ABSORB_NONE && c->d.absorb_cells > 0)
                    ? std::max(0, c->G.nr - c->G.absorb_cells - 1) : -1;
}

void ens_filter(const EnsFieldArg *tab, const EnsList &L, int blocks, int pass, cudaStream_t s) {
  k_ens_filter<<<(unsigned)blocks, 256, 0, s>>>(tab, L, pass);
}
void ens_b_half(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s) {
  k_ens_b_half<<<(unsigned)blocks, 256, 0, s>>>(tab, L);
}
void ens_e_full(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s) {
  k_ens_e_full<<<(unsigned)blocks, 256, 0, s>>>(tab, L);
}
void ens_lossy(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s) {
  k_ens_lossy<<<(unsigned)blocks, 256, 0, s>>>(tab, L);
}
void ens_ghosts(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s) {
  k_ens_ghosts<<<(unsigned)blocks, 256, 0, s>>>(tab, L);
}
void ens_copy32(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s) {
  k_ens_copy32<<<(unsigned)blocks, 256, 0, s>>>(tab, L);
}
void ens_inject_sigma(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s) {
  k_ens_sigma<<<(unsigned)blocks, 256, 0, s>>>(tab, L);
}
void ens_inject_smooth(const EnsFieldArg *tab, const EnsList &L, int blocks, int pass, cudaStream_t s) {
  k_ens_smooth<<<(unsigned)blocks, 256, 0, s>>>(tab, L, pass);
}
void ens_inject_write(const EnsFieldArg *tab, const EnsList &L, int blocks, cudaStream_t s) {
  k_ens_write<<<(unsigned)blocks, 256, 0, s>>>(tab, L);
}

void fields_b_half(pic_ctx *c) {
  const Grid &G = c->G;
  ++c->launches, k_b_half<<<grid2(G.nr + 1, G.nth + 1), dim3(BX, BY), 0, c->stream>>>(G, c->f[ER], c->f[ETH], c->f[EPH], c->f[BR],
                                                                      c->f[BTH], c->f[BPH]);
}

void fields_e_full(pic_ctx *c) {
  const Grid &G = c->G;
  ++c->launches, k_e_full<<<grid2(G.nr + 1, G.nth + 1), dim3(BX, BY), 0, c->stream>>>(
      G, c->f[ER], c->f[ETH], c->f[EPH], c->f[BR], c->f[BTH], c->f[BPH], c->F[0], c->F[1], c->F[2]);
}

void fields_copy32(pic_ctx *c) {
  const Grid &G = c->G;
  ++c->launches, k_copy32<<<grid2(G.nr + 2 * G.g + 1, G.nth + 2), dim3(BX, BY), 0, c->stream>>>(
      G, c->f[0], c->f[1], c->f[2], c->f[3], c->f[4], c->f[5], c->f32[0], c->f32[1], c->f32[2], c->f32[3], c->f32[4],
      c->f32[5]);
}

void fields_fill_ghosts(pic_ctx *c) {
  const Grid &G = c->G;
  ++c->launches, k_axis_ghosts<<<(G.nr + 1 + 127) / 128, 128, 0, c->stream>>>(G, c->f[ETH], c->f[BR], c->f[BPH]);
  if (c->d.precision == PIC_FP32) fields_copy32(c);
}

void fields_finish(pic_ctx *c) {
  const Grid &G = c->G;
  if (c->d.absorb_profile != PIC_ABSORB_NONE && c->d.absorb_cells > 0) {
    int i0 = G.nr - G.absorb_cells - 1;
    if (i0 < 0) i0 = 0;
    ++c->launches, k_lossy<<<grid2(G.nr + 1 - i0, G.nth + 1), dim3(BX, BY), 0, c->stream>>>(G, c->f[0], c->f[1], c->f[2], c->f[3],
                                                                           c->f[4], c->f[5], i0);
  }
  fields_fill_ghosts(c);
}

void filter_array(pic_ctx *c, double *a, double *tmp, int half_j, int sign, int passes) {
  (void)sign;  // the fold sign is built into the weights of k_filter
  const Grid &G = c->G;
  dim3 gr = grid2(G.nr + 2 * G.g + 1, G.nth + 1);
  double *src = a, *dst = tmp;
  for (int p = 0; p < passes; ++p) {
    ++c->launches, k_filter<<<gr, dim3(BX, BY), 0, c->stream>>>(G, src, dst, half_j);
    double *t = src; src = dst; dst = t;
  }
  if (src != a)
    cudaMemcpyAsync(a, src, c->grid_elems * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
}

void fields_filter(pic_ctx *c) {
  const int n = c->d.n_filt;
  if (n <= 0) return;
  const Grid &G = c->G;
  dim3 gr = grid2(G.nr + 2 * G.g + 1, G.nth + 1);
  for (int p = 0; p < n; ++p) {
    for (int k = 0; k < 3; ++k)
      ++c->launches, k_filter<<<gr, dim3(BX, BY), 0, c->stream>>>(G, c->F[k], c->Ft[k], k == 1);
    for (int k = 0; k < 3; ++k) { double *t = c->F[k]; c->F[k] = c->Ft[k]; c->Ft[k] = t; }
  }
}

void inject(pic_ctx *c, double t) {
  const Grid &G = c->G;
  const int npp = c->d.pairs_per_cell, ns = c->d.inject_smooth;
  long long *smax = c->d_cnt + CNT_SMAX;
  cudaMemsetAsync(smax, 0, sizeof(long long), c->stream);
  double *a = c->sig, *b = c->sig + (G.nth + 1);
  const int tb = (G.nth + 127) / 128;
  ++c->launches, k_inject_sigma<<<tb, 128, 0, c->stream>>>(G, c->f[ER], t, a, ns ? nullptr : smax);
  for (int p = 0; p < ns; ++p) {
    ++c->launches, k_inject_smooth<<<tb, 128, 0, c->stream>>>(G.nth, a, b, p == ns - 1 ? smax : nullptr);
    double *x = a; a = b; b = x;
  }
  const InjectRule R{c->d.inject, npp, c->d.f_inj, c->d.inject_q, c->d.inject_seed, (uint64_t)c->step};
  const int64_t nslots = (int64_t)G.nth * npp * 2;
  const int blocks = (int)((nslots + 255) / 256);
  if (c->d.precision == PIC_FP32)
    ++c->launches, k_inject_write<true><<<blocks, 256, 0, c->stream>>>(G, a, smax, c->p64, c->p32, c->n_used, c->next_id, R,
                                                        c->d_cnt + CNT_INJECTED, c->d_cnt + CNT_CAPPED, c->qexp);
  else
    ++c->launches, k_inject_write<false><<<blocks, 256, 0, c->stream>>>(G, a, smax, c->p64, c->p32, c->n_used, c->next_id, R,
                                                         c->d_cnt + CNT_INJECTED, c->d_cnt + CNT_CAPPED, c->qexp);
  c->n_used += nslots;
  c->next_id += nslots;
}

// Spin-down luminosity (Sec. 5.3, Fig. 7d): the radial Poynting flux
// (E x B)_r of the total field, plasma plus analytic at time t, through the
// sphere of node radius r_i, one block per interior row.  On the sphere the
// meridional cell j carries E_th(i, j+1/2); B_ph (at i -+ 1/2), E_ph (at the
// nodes j, j+1) and B_th (at i -+ 1/2 and j, j+1) are averaged to the cell's
// centre; each cell adds (E_th B_ph - E_ph B_th) 2 pi r_i^2 (cos th_j -
// cos th_{j+1}).  L[0] and L[nr] are 0.
__global__ void k_luminosity(Grid G, const double *__restrict__ Et, const double *__restrict__ Ep,
                             const double *__restrict__ Bt, const double *__restrict__ Bp, double t, double *L) {
  __shared__ double sm[32];
  const Metric &m = G.m;
  const int i = blockIdx.x;
  double s = 0.0;
  if (i >= 1 && i < G.nr) {
    const double r = m.r_n[i + G.PI], ring = 2.0 * PI_D * r * r;
    const Vac<double> V{G.vacuum, G.b0, G.r_min, omega_at(G.omega, G.t_spin, t)};
    for (int j = threadIdx.x; j < G.nth; j += blockDim.x) {
      const int cj = j + G.PJ;
      double E[3], B[3];
      vacuum_field<double>(V, r, m.sin_tb[cj], m.cos_tb[cj], false, E, B);
      const size_t o = gidx(G, i, j);
      const double et = Et[o] + E[1];
      const double bp = 0.5 * (Bp[o - G.LD] + Bp[o]) + B[2];
      const double ep = 0.5 * (Ep[o] + Ep[o + 1]) + E[2];
      const double bt = 0.25 * (Bt[o - G.LD] + Bt[o] + Bt[o - G.LD + 1] + Bt[o + 1]) + B[1];
      s += (et * bp - ep * bt) * ring * m.vol_t_h[cj];
    }
  }
  for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sm[w];
    L[i] = tot;
  }
}

void luminosity(pic_ctx *c, double t, double *L) {
  const Grid &G = c->G;
  ++c->launches, k_luminosity<<<G.nr + 1, 256, 0, c->stream>>>(G, c->f[ETH], c->f[EPH], c->f[BTH], c->f[BPH], t, L);
}

void gauss_rows(pic_ctx *c, int ilo, int imax, bool snapshot) {
  const Grid &G = c->G;
  if (imax < ilo) return;
  ++c->launches, k_gauss<<<grid2(imax - ilo + 1, G.nth + 1), dim3(BX, BY), 0, c->stream>>>(
      G, c->f[ER], c->f[ETH], c->Q, c->Qa, c->gsnap, ilo, imax, snapshot ? 1 : 0, c->d_cnt + CNT_GMAX,
      c->d_cnt + CNT_QMAX);
}

void field_energy_rows(pic_ctx *c, int imax) {
  const Grid &G = c->G;
  ++c->launches, k_field_energy<<<grid2(G.nr + 1, G.nth + 1), dim3(BX, BY), 0, c->stream>>>(
      G, c->f[0], c->f[1], c->f[2], c->f[3], c->f[4], c->f[5], imax, c->d_acc + ACC_FIELD);
}

void moments(pic_ctx *c, bool snapshot, pic_moments *out) {
  const Grid &G = c->G;
  cudaMemsetAsync(c->Q, 0, c->grid_elems * sizeof(double), c->stream);
  cudaMemsetAsync(c->Qa, 0, c->grid_elems * sizeof(double), c->stream);
  if (c->d.precision == PIC_FP32) charge32(c, c->Q, c->Qa);
  else charge64(c, c->Q, c->Qa);
  filter_array(c, c->Q, c->Qt, 0, +1, c->d.n_filt);
  int L = c->d.absorb_profile == PIC_ABSORB_NONE ? 0 : c->d.absorb_cells;
  int imax = G.nr - L - 1;
  cudaMemsetAsync(c->d_cnt + CNT_GMAX, 0, 2 * sizeof(long long), c->stream);
  if (imax >= 1)
    ++c->launches, k_gauss<<<grid2(imax, G.nth + 1), dim3(BX, BY), 0, c->stream>>>(G, c->f[ER], c->f[ETH], c->Q, c->Qa, c->gsnap,
                                                                    1, imax, snapshot ? 1 : 0, c->d_cnt + CNT_GMAX,
                                                                    c->d_cnt + CNT_QMAX);
  if (snapshot) { c->have_snap = true; return; }
  cudaMemsetAsync(c->d_acc, 0, ACC_N * sizeof(double), c->stream);
  cudaMemsetAsync(c->d_cnt + CNT_LIVE, 0, sizeof(long long), c->stream);
  ++c->launches, k_field_energy<<<grid2(G.nr + 1, G.nth + 1), dim3(BX, BY), 0, c->stream>>>(
      G, c->f[0], c->f[1], c->f[2], c->f[3], c->f[4], c->f[5], G.nr, c->d_acc + ACC_FIELD);
  if (c->d.precision == PIC_FP32) reduce_particles32(c);
  else reduce_particles64(c);
  long long cnt[CNT_N];
  double acc[ACC_N];
  cudaMemcpyAsync(cnt, c->d_cnt, sizeof cnt, cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(acc, c->d_acc, sizeof acc, cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  double gmax, qmax;
  memcpy(&gmax, &cnt[CNT_GMAX], sizeof(double));
  memcpy(&qmax, &cnt[CNT_QMAX], sizeof(double));
  out->live = cnt[CNT_LIVE];
  out->deleted = cnt[CNT_DELETED];
  out->injected = cnt[CNT_INJECTED];
  out->inject_capped = cnt[CNT_CAPPED];
  out->axis_ties = cnt[CNT_TIES];
  out->step = c->step;
  out->dt = G.dt;
  out->time = c->step * G.dt;
  out->kinetic_energy = acc[ACC_KIN];
  out->field_energy = acc[ACC_FIELD];
  out->total_charge = acc[ACC_CHARGE];
  out->gauss_residual = (!c->have_snap) ? -1.0 : (qmax > 0 ? gmax / qmax : gmax);
}

}  // namespace pic

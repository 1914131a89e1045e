// count_impl.cuh -- kernel body of the pair counter, instantiated per kind
// in count_mono.cu, count_sigpi.cu and count_rmu.cu.
//
// Three accumulation policies share the traversal and the binning:
//   kAccCount    -- pair counts (Sec. 2.2 Eq. 11);
//   kAccWeighted -- counts and, per bin, the sum of w_i w_j (the pixel and
//                   density-grid weights of Sec. 3.4);
//   kAccAdjoint  -- d/dw_i of sum_b G_b W_b = sum_j w_j G[bin(i, j)] for
//                   every home object i (no counts);
//   kAccIntWeighted -- counts and weight sums for integer weights, in
//                   integer histograms (monopole and chord counts).
#pragma once

#include "count_kernel.cuh"

#include <algorithm>
#include <type_traits>
#include <atomic>

namespace cute {

constexpr int kAccCount = 0, kAccWeighted = 1, kAccAdjoint = 2;
// integer weights (all weights integers in [0, 2048], e.g. counts per pixel):
// counts, and the weight products w_i w_j -- exact integers below 2^22 -- in
// a second uint32 histogram, flushed to FP64 as exact sums
constexpr int kAccIntWeighted = 3;

template <int HP>
struct Home {
  static_assert(HP % 2 == 0, "home slots come in pairs (packed FP32 math)");
  // slots 2k and 2k+1 share a float2 (packed math); scalar access by slot
  float2 nx2[HP / 2], ny2[HP / 2], nz2[HP / 2];  // -(home position - image shift), grid frame
  float2 nq2[HP / 2];                            // R_MU: -q_i, q_i = |x_i|^2 - q0
  float2 c2[HP / 2];                             // R_MU: k (2 q_i + 4 q0)
  float w[HP];                 // weight (0 when padded)
  float gh[HP], gl[HP];        // adjoint: float-float gradient accumulator
  int id[HP];                  // sorted index in A (INT_MAX when padded)
  __device__ __forceinline__ static float get(const float2 *a, int s) {
    return (s & 1) ? a[s >> 1].y : a[s >> 1].x;
  }
  __device__ __forceinline__ static void put(float2 *a, int s, float v) {
    if (s & 1) a[s >> 1].y = v; else a[s >> 1].x = v;
  }
};

struct WarpSmem {
  int gje;                     // end of the current item's neighbour range
  uint32_t *hist;
  uint32_t *whist;             // integer weights: the weight-product histogram
  uint32_t s_dw;               // its byte offset from the count histogram
  char *hist_lane;
  uint32_t s_hist_lane;        // shared-space address of hist_lane
  uint32_t s_wcol;             // shared-space address of wcol
  uint32_t s_G;                // shared-space address of G
  float2 *wcol;                // weighted: this lane's float-float column
  float2 *wall;                // weighted: all columns of the warp
  int wstride;                 // weighted: float2 entries per column
  const float2 *G;             // adjoint: G per slot, float-float
  int *qcnt;
  int2 *queue;
  int qcap;
  float4 *tiles;
  float *wtiles;               // R_MU weighted / adjoint: the tiles' weights
  uint32_t s_box;              // the item's home box, negated: (-lo.xyz, carried rows),
                               // (-hi.xyz, end of the run's real rows)
  uint32_t s_cidx;             // neighbour index of each culled row, by row of the
                               // tile buffer (INT_MAX: padding row)
};

// ------------------------------------------------------------------ float-float
// The pair (hi, lo) represents hi + lo.  (hi, lo) += (ph + pl): Knuth's
// TwoSum (df_stage.h), then Dekker/Kahan's FastTwoSum to renormalise.
__device__ __forceinline__ void ff_add(float &hi, float &lo, float ph, float pl) {
  float s, e;
  dfs::two_sum(hi, ph, s, e);
  const float t = __fadd_rn(lo, __fadd_rn(e, pl));
  hi = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(hi, s));
}

// ------------------------------------------------------------------ queue
// Warp-cooperative re-test of queued pairs, 32 at a time (all of them when
// draining): the double-float stage, then the FP64 formula for the pairs
// it leaves open.  Every lane must call it.
template <int KIND, int ACC>
__device__ __forceinline__ void process_queue(const KParams &p, const PairDev &pd, const WarpSmem &w,
                                           int lane, bool drain) {
  __syncwarp();
  int n = *w.qcnt;
  int done = 0;
  unsigned fp64 = 0;
  const int nb = p.n0 * p.n1;
  while (n >= 32 || (drain && n > 0)) {
    int take = min(n, 32);
    if (lane < take) {
      int2 e = w.queue[n - take + lane];
      int s;
      if (!slot_df<KIND>(p, pd, e.x, e.y, s)) {
        s = slot64<KIND>(p, pd, e.x, e.y);
        fp64++;
      }
      int s0 = s / p.slots1, s1 = s - s0 * p.slots1;
      bool in = s0 >= 1 && s0 <= p.n0 && (p.slots1 == 1 || (s1 >= 1 && s1 <= p.n1));
      int b = (s0 - 1) * p.n1 + (p.slots1 == 1 ? 0 : s1 - 1);
      if (ACC != kAccAdjoint) atomicAdd(&w.hist[s * p.R + (lane & (p.R - 1))], 1u);
      if ((ACC == kAccWeighted || ACC == kAccIntWeighted) && in) {
        double prod = (double)pd.posA[e.x].w * (double)pd.posB[e.y].w;  // exact
        atomicAdd(&p.out_wsum[(size_t)pd.out * nb + b], prod);
      }
      if (ACC == kAccAdjoint && in) {
        double t = (double)pd.posB[e.y].w * p.G[b];
        atomicAdd(&p.grad[pd.permA[e.x]], t);
      }
    }
    n -= take;
    done += take;
  }
  __syncwarp();
  if (fp64) atomicAdd(&p.stats[5], (unsigned long long)fp64);
  if (lane == 0) {
    *w.qcnt = n;
    if (done) atomicAdd(&p.stats[0], (unsigned long long)done);
  }
  __syncwarp();
}

// add the warp's histogram to output `out` in HBM and clear it
static __device__ __forceinline__ void flush_hist(const KParams &p, const WarpSmem &w, int out, int lane) {
  __syncwarp();
  const int nb = p.n0 * p.n1;
  for (int b = lane; b < nb; b += 32) {
    int b0 = b / p.n1, b1 = b - b0 * p.n1;
    int s = (b0 + 1) * p.slots1 + (p.slots1 > 1 ? b1 + 1 : 0);
    unsigned long long sum = 0;
    for (int r = 0; r < p.R; r++) sum += w.hist[s * p.R + r];
    if (sum) atomicAdd(&p.out_counts[(size_t)out * nb + b], sum);
  }
  __syncwarp();
  for (int i = lane; i < p.nslots * p.R; i += 32) w.hist[i] = 0;
  __syncwarp();
}

// integer weights: add the warp's weight-product histogram to output `out`
// (exact: a uint64 sum of integers, below 2^53) and clear it
static __device__ __forceinline__ void flush_whist(const KParams &p, const WarpSmem &w, int out,
                                                   int lane) {
  __syncwarp();
  const int nb = p.n0 * p.n1;
  for (int b = lane; b < nb; b += 32) {
    int b0 = b / p.n1, b1 = b - b0 * p.n1;
    int s = (b0 + 1) * p.slots1 + (p.slots1 > 1 ? b1 + 1 : 0);
    unsigned long long sum = 0;
    for (int r = 0; r < p.R; r++) sum += w.whist[s * p.R + r];
    if (sum) atomicAdd(&p.out_wsum[(size_t)out * nb + b], (double)sum);
  }
  __syncwarp();
  for (int i = lane; i < p.nslots * p.R; i += 32) w.whist[i] = 0;
  __syncwarp();
}

// add the warp's float-float weighted columns to output `out` and clear them
static __device__ __forceinline__ void flush_wsum(const KParams &p, const WarpSmem &w, int out,
                                               int lane) {
  __syncwarp();
  const int nb = p.n0 * p.n1;
  for (int b = lane; b < nb; b += 32) {
    int b0 = b / p.n1, b1 = b - b0 * p.n1;
    int s = (b0 + 1) * p.slots1 + (p.slots1 > 1 ? b1 + 1 : 0);
    float hi = 0.0f, lo = 0.0f;
    for (int c = 0; c < 32; c++) {
      const float2 v = w.wall[c * w.wstride + s];
      ff_add(hi, lo, v.x, v.y);
    }
    const double sum = (double)hi + (double)lo;
    if (sum != 0.0) atomicAdd(&p.out_wsum[(size_t)out * nb + b], sum);
  }
  __syncwarp();
  for (int i = lane; i < 32 * w.wstride; i += 32) w.wall[i] = make_float2(0.0f, 0.0f);
  __syncwarp();
}

// ------------------------------------------------------------------ binning
// Table binning (non-uniform edges): slot byte offset (slot * R * 4) of one
// pair from its FP32 values -- the squared separation v (monopole, theta),
// sigma^2 and pi^2, or r^2 and mu -- and whether it lies inside an edge's
// FP32 error band (then it is re-tested).
template <int KIND, int M0, int M1>
__device__ __forceinline__ uint32_t table_slot(const KParams &p, uint32_t lut, uint32_t band,
                                               float a, float b, bool &near) {
  const uint32_t stride0 = (uint32_t)p.slots1 * p.R * 4u, stride1 = (uint32_t)p.R * 4u;
  if (KIND == KMONO || KIND == KTHETA) {
    const uint32_t e0 = lut_get<M0>(lut, p.ax[0], a);
    return axis_resolve(band, p.ax[0], a, e0, stride0, near);
  } else if (KIND == KSIGPI) {
    const uint32_t e0 = lut_get<M0>(lut, p.ax[0], a);
    const uint32_t e1 = lut_get<M1>(lut, p.ax[1], b);
    bool n0, n1;
    const uint32_t o = axis_resolve(band, p.ax[0], a, e0, stride0, n0) +
                       axis_resolve(band, p.ax[1], b, e1, stride1, n1);
    near = n0 || n1;
    return o;
  } else {
    const uint32_t e0 = lut_get<M0>(lut, p.ax[0], a);
    const uint32_t e1 = lut_get<M1>(lut, p.ax[1], b);
    // the mu bound of the pair's r slot: class c scales the base by 2^c
    const float eps = __int_as_float(__float_as_int(p.mu_eps_base) +
                                     (int)(((e0 >> kClassShift) & 0xFu) << 23));
    bool n0, n1;
    const uint32_t o = axis_resolve(band, p.ax[0], a, e0, stride0, n0) +
                       mu_resolve(band, p.ax[1], b, e1, stride1, eps, n1);
    near = n0 || n1;
    return o;
  }
}

// (r, mu) values of two pairs in packed FP32: s = x_j - x_i, r^2 = s.s
// (floored at 1e-30, so 1/r and mu stay finite); with l = x_i + x_j and the
// per-object q = |x|^2 - q0 (observer frame), s.l = |x_j|^2 - |x_i|^2 =
// q_j - q_i and l.l = 2|x_i|^2 + 2|x_j|^2 - r^2, formed scaled by k:
// k l.l = k (2 q_j) + (k (2 q_i + 4 q0) - k r^2).  Then
// |s.l| / sqrt(r^2 k l.l) = mu / sqrt(k).
struct Rmu2 {
  float2 r2, sl, l2;  // r^2, s.l, k l.l
};
__device__ __forceinline__ Rmu2 rmu_values2(float2 qx, float2 qy, float2 qz, float2 qq, float2 nx,
                                            float2 ny, float2 nz, float2 nqi, float2 ci,
                                            float2 k2, float2 nk) {
  const float2 dx = __fadd2_rn(qx, nx), dy = __fadd2_rn(qy, ny), dz = __fadd2_rn(qz, nz);
  Rmu2 v;
  v.r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, make_float2(kVFloor, kVFloor))));
  v.sl = __fadd2_rn(qq, nqi);
  v.l2 = __ffma2_rn(qq, k2, __ffma2_rn(v.r2, nk, ci));
  return v;
}

// Uniform edges, two home objects at once with the packed FP32 instructions
// of sm_100+ (element-wise IEEE round-to-nearest: each element is rounded
// as the scalar formula would be).  Each gives the byte offsets of the two
// pairs' slots and a near score per pair: the pair lies inside an edge's
// error band (and is re-tested) when its score reaches the kind's
// threshold, near_thr.  Monopole (and theta on chords):
__device__ __forceinline__ void mono_arith2(const AxisPlan &a, float2 qx, float2 qy, float2 qz,
                                            float2 nx, float2 ny, float2 nz, uint32_t stride,
                                            uint32_t c, uint32_t &o0, uint32_t &o1, float2 &sc) {
  const float2 dx = __fadd2_rn(qx, nx), dy = __fadd2_rn(qy, ny), dz = __fadd2_rn(qz, nz);
  // v >= 1e-30 (a floor far below any nonzero squared separation of FP32
  // coordinates), so x = v / sqrt(v) is finite and t >= -1/2
  const float2 v = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, make_float2(kVFloor, kVFloor))));
  const float2 x = __fmul2_rn(v, make_float2(rsqrt_hw(v.x), rsqrt_hw(v.y)));
  float2 t = __ffma2_rn(x, make_float2(a.inv, a.inv), make_float2(a.cst, a.cst));
  t.x = fminf(t.x, a.thi);  // above the last edge (and far sentinels): the top slot
  t.y = fminf(t.y, a.thi);
  const float2 tm = __fadd2_rn(t, make_float2(kMagic, kMagic));
  const float2 fl = __fadd2_rn(tm, make_float2(-kMagic, -kMagic));
  const float2 h = __ffma2_rn(fl, make_float2(-1.0f, -1.0f), t);  // t - floor, exact
  sc = make_float2(fabsf(h.x), fabsf(h.y));  // near when >= near_at
  o0 = __float_as_uint(tm.x) * stride + c;
  o1 = __float_as_uint(tm.y) * stride + c;
}

// Log-spaced edges (kArithLog), monopole and chords, two pairs at once:
// v clamped below at vlo (where t = -1: slot 0), t = A log2(v) +
// (D v + B) v + C by the hardware log2 (PTX lg2.approx.ftz.f32), clamped
// above to thi; the pair is near an edge when |h| + thr_a / sqrt(v)
// reaches near_c (the bound falls as 1/sqrt(v); one FMA per pair).
__device__ __forceinline__ float lg2_hw(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
template <bool CLAMP>
__device__ __forceinline__ void mono_log2(const AxisPlan &a, float2 qx, float2 qy, float2 qz,
                                          float2 nx, float2 ny, float2 nz, uint32_t stride,
                                          uint32_t c, uint32_t &o0, uint32_t &o1, float2 &sc) {
  const float2 dx = __fadd2_rn(qx, nx), dy = __fadd2_rn(qy, ny), dz = __fadd2_rn(qz, nz);
  float2 v = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
  v.x = fmaxf(v.x, a.vlo);
  v.y = fmaxf(v.y, a.vlo);
  const float2 lg = make_float2(lg2_hw(v.x), lg2_hw(v.y));
  const float2 rr = make_float2(rsqrt_hw(v.x), rsqrt_hw(v.y));
  const float2 pv = __ffma2_rn(v, __ffma2_rn(v, make_float2(a.ld, a.ld), make_float2(a.lb, a.lb)),
                               make_float2(a.cst, a.cst));
  float2 t = __ffma2_rn(lg, make_float2(a.inv, a.inv), pv);
  if (CLAMP) {  // above the last edge (and far sentinels): the top slot
    t.x = fminf(t.x, a.thi);
    t.y = fminf(t.y, a.thi);
  }  // (kArithLogU: the spare slots above the last bin hold every t)
  const float2 tm = __fadd2_rn(t, make_float2(kMagic, kMagic));
  const float2 fl = __fadd2_rn(tm, make_float2(-kMagic, -kMagic));
  const float2 h = __ffma2_rn(fl, make_float2(-1.0f, -1.0f), t);
  sc = make_float2(fmaf(rr.x, a.thr_a, fabsf(h.x)), fmaf(rr.y, a.thr_a, fabsf(h.y)));
  o0 = __float_as_uint(tm.x) * stride + c;
  o1 = __float_as_uint(tm.y) * stride + c;
}

// Two (r, mu) pairs at once with uniform edges on both axes.
__device__ __forceinline__ float2 clampt(float2 t, float hi) {
  return make_float2(fminf(t.x, hi), fminf(t.y, hi));
}
__device__ __forceinline__ void rmu_arith2(const AxisPlan &a0, const AxisPlan &a1, float2 qx,
                                           float2 qy, float2 qz, float2 qq, float2 nx, float2 ny,
                                           float2 nz, float2 nqi, float2 ci, float2 k2, float2 nk,
                                           float sl1, uint32_t stride1, uint32_t c,
                                           uint32_t &o0, uint32_t &o1, float2 &sc) {
  const Rmu2 v = rmu_values2(qx, qy, qz, qq, nx, ny, nz, nqi, ci, k2, nk);
  const float2 r2 = v.r2, sl = v.sl, l2 = v.l2;
  const float2 rr = make_float2(rsqrt_hw(r2.x), rsqrt_hw(r2.y));
  // k l.l is positive for every pair within reach; a candidate beyond it
  // (or a padded slot, whose k l.l is negative) may give a NaN, which the
  // clamp below turns into the top slot
  const float2 pl = __fmul2_rn(r2, l2);
  // t >= -1/2 on both axes (e_0 = 0); clamped above only.  Axis 1: the
  // scale k = 1/inv^2 makes |s.l| rsqrt(r^2 k l.l) = mu inv (cst + mu inv in
  // one FMA)
  const float2 t0 = clampt(__ffma2_rn(__fmul2_rn(r2, rr), make_float2(a0.inv, a0.inv),
                                      make_float2(a0.cst, a0.cst)), a0.thi);
  const float2 t1 = clampt(__ffma2_rn(make_float2(fabsf(sl.x), fabsf(sl.y)),
                                      make_float2(rsqrt_hw(pl.x), rsqrt_hw(pl.y)),
                                      make_float2(a1.cst, a1.cst)),
                           a1.thi);
  const float2 m2 = make_float2(kMagic, kMagic), nm2 = make_float2(-kMagic, -kMagic),
               neg = make_float2(-1.0f, -1.0f);
  const float2 tm0 = __fadd2_rn(t0, m2), tm1 = __fadd2_rn(t1, m2);
  const float2 f0 = __fadd2_rn(tm0, nm2);                        // rint(t0)
  const float2 h0 = __ffma2_rn(f0, neg, t0);                     // t - rint(t), exact
  const float2 h1 = __ffma2_rn(__fadd2_rn(tm1, nm2), neg, t1);
  // magic + rint(t0) * slots1 + rint(t1): exact (an integer below 2^24)
  const float2 tc = __ffma2_rn(f0, make_float2(sl1, sl1), tm1);
  // near an edge: |h| within the error bound of 1/2 on either axis (the mu
  // bound thr_a / r + thr_b, with the 1/r that rr already holds): the score
  // max(|h0|, |h1| + thr_a rr) reaches min(near_at, near_c) (one FMA, its
  // rounding covered by near_c's 2^-22 margin)
  sc = make_float2(fmaxf(fabsf(h0.x), fmaf(rr.x, a1.thr_a, fabsf(h1.x))),
                   fmaxf(fabsf(h0.y), fmaf(rr.y, a1.thr_a, fabsf(h1.y))));
  o0 = __float_as_uint(tc.x) * stride1 + c;
  o1 = __float_as_uint(tc.y) * stride1 + c;
}

// Two (sigma, pi) pairs at once with uniform edges on both axes (near when
// |h| reaches near_at on either axis, pi's |h| rescaled to sigma's).
__device__ __forceinline__ void sigpi_arith2(const AxisPlan &a0, const AxisPlan &a1, float2 qx,
                                             float2 qy, float2 qz, float2 nx, float2 ny,
                                             float2 nz, float sl1, uint32_t stride1,
                                             uint32_t c, uint32_t &o0, uint32_t &o1, float2 &sc) {
  const float2 dx = __fadd2_rn(qx, nx), dy = __fadd2_rn(qy, ny), dz = __fadd2_rn(qz, nz);
  const float2 v0 = __ffma2_rn(dy, dy, __ffma2_rn(dx, dx, make_float2(kVFloor, kVFloor)));
  const float2 x0 = __fmul2_rn(v0, make_float2(rsqrt_hw(v0.x), rsqrt_hw(v0.y)));
  const float2 t0 = clampt(__ffma2_rn(x0, make_float2(a0.inv, a0.inv), make_float2(a0.cst, a0.cst)),
                           a0.thi);
  const float2 t1 = clampt(__ffma2_rn(make_float2(fabsf(dz.x), fabsf(dz.y)),
                                      make_float2(a1.inv, a1.inv), make_float2(a1.cst, a1.cst)),
                           a1.thi);
  const float2 m2 = make_float2(kMagic, kMagic), nm2 = make_float2(-kMagic, -kMagic),
               neg = make_float2(-1.0f, -1.0f);
  const float2 tm0 = __fadd2_rn(t0, m2), tm1 = __fadd2_rn(t1, m2);
  const float2 f0 = __fadd2_rn(tm0, nm2);
  const float2 h0 = __ffma2_rn(f0, neg, t0);
  const float2 h1 = __ffma2_rn(__fadd2_rn(tm1, nm2), neg, t1);
  const float2 tc = __ffma2_rn(f0, make_float2(sl1, sl1), tm1);  // as for (r, mu)
  // pi's |h| scaled to sigma's threshold (rounded up: never fewer flags)
  const float2 g1 = __fmul2_rn(h1, make_float2(a1.near_scale, a1.near_scale));
  sc = make_float2(fmaxf(fabsf(h0.x), fabsf(g1.x)), fmaxf(fabsf(h0.y), fabsf(g1.y)));
  o0 = __float_as_uint(tc.x) * stride1 + c;
  o1 = __float_as_uint(tc.y) * stride1 + c;
}

// Stores two pairs' slot offsets and near scores from the arithmetic
// binning: pairs that are not pairs of this item (MASK) go to the unused
// slot 0 with score 0; without the lazy count, near pairs also go to
// slot 0 and are marked in nmask at once.
template <int HP, int MASK, bool LAZY, int NP>
__device__ __forceinline__ void arith_pair_out(float2 s2, uint32_t (&o)[2], int u, int sp, int gj,
                                               const Home<HP> &h, uint32_t zoff, float thr,
                                               uint32_t (&off)[NP], float (&sc)[NP],
                                               unsigned &nmask) {
#pragma unroll
  for (int e = 0; e < 2; e++) {
    const int s = 2 * sp + e, k = u * HP + s;
    float v = e ? s2.y : s2.x;
    if (MASK == 1 && !(gj > h.id[s])) { o[e] = zoff; v = 0.0f; }
    if (MASK == 2 && gj == h.id[s]) { o[e] = zoff; v = 0.0f; }
    if (!LAZY && v >= thr) { o[e] = zoff; nmask |= 1u << k; }
    off[k] = o[e];
    sc[k] = v;
  }
}

// Score threshold of the arithmetic binning: |h| >= near_at of axis 0
// (monopole, theta; sigma, pi with pi rescaled), or the smaller of near_at
// of r and near_c of mu (r, mu: a few more flags than the exact per-axis
// tests, all decided by the re-test).
template <int KIND, int M0>
__device__ __forceinline__ float near_thr(const KParams &p) {
  if (M0 == kArithLog || M0 == kArithLogU) return p.ax[0].near_c;
  if (KIND == KRMU) return fminf(p.ax[0].near_at, p.ax[1].near_c);
  return p.ax[0].near_at;
}

// All pairs of the HP home objects of each lane with the cnt neighbours of
// one shared-memory tile (cnt even; rows past the slice hold sentinels).
// Two neighbours at a time: every binning of the 2 x HP pairs is issued
// first, then the accumulation; pairs inside an edge's error band go to the
// warp's re-test queue (rare, so the enqueue sits behind one vote).  With
// arithmetic binning every pair goes to the slot its FP32 value gives and
// the warp votes on the step's largest near score; a flagged step (rare)
// takes the near pairs' contributions back (count, weight product or
// gradient term) before queueing them, so the common step carries no
// per-pair selects.  Table binning routes near pairs to slot 0 at once.
// MASK: 0 -- every pair counts; the rows are culled rows of a tile buffer
//            from its row gj0 on (their neighbour indices in s_cidx or
//            the rows' weight words, the end of the real rows in the box
//            words);
//       1 -- only j > i counts (the home run against itself, unique pairs);
//       2 -- every j != i counts (full-stencil adjoint of an auto count).
// R_MU tiles hold (x, y, z, q); their weights (weighted, adjoint) come
// from a tile of their own, wtile.
template <int KIND, int HP, int M0, int M1, int MASK, int ACC>
__device__ __forceinline__ void tile_pairs(const KParams &p, uint32_t lut, uint32_t band,
                                           const PairDev &pd, const WarpSmem &w, uint32_t tile,
                                           uint32_t wtile, int cnt, int gj0, Home<HP> &h,
                                           int lane, unsigned &near_count) {
  constexpr int U = 8 / HP;  // neighbours per step: 8 pairs per lane per step
  constexpr int NP = U * HP;
  constexpr bool kLazy = M0 == kArith || M0 == kArithLog || M0 == kArithLogU;
  const float thr = near_thr<KIND, M0>(p);
  const int slot_shift = 31 - __clz(p.R * 4);
  // Plain counts add straight to the lane's histogram copy: its shared
  // address is folded into the offset constants (slot k = bits - magic + 1
  // on each axis), and a pair that is not counted here goes to slot 0
  // (below range, never reported).
  constexpr bool kDirect = ACC == kAccCount || ACC == kAccIntWeighted;  // offsets are addresses
  // culled rows of plain counts but (r, mu) carry their neighbour index in
  // the weight word (unused there); the others keep it in s_cidx
  constexpr bool kIdxRow = ACC == kAccCount && KIND != KRMU;
  const uint32_t zoff = kDirect ? w.s_hist_lane : 0u;
  const uint32_t st0 = (uint32_t)p.slots1 * p.R * 4u, st1 = (uint32_t)p.R * 4u;
  const uint32_t c1d = (1u - kMagicBits) * st0 + zoff;
  // 2-D: slot (rint(t0) + 1) * slots1 + rint(t1) + 1 from the bits of
  // magic + rint(t0) * slots1 + rint(t1)
  const float sl1 = (float)p.slots1;
  const uint32_t c2d = ((uint32_t)p.slots1 + 1u - kMagicBits) * st1 + zoff;
  // R_MU: k l.l = 2k q_j + (C_i - k r^2)
  const float lk = p.ax[1].lsc;
  const float2 k2 = make_float2(2.0f * lk, 2.0f * lk), nk = make_float2(-lk, -lk);
  for (int j = 0; j < cnt; j += U) {
    uint32_t off[NP];
    float sc[NP];  // arithmetic binning: near scores
    float wj[U];
    unsigned nmask = 0;
#pragma unroll
    for (int u = 0; u < U; u++) {
      const float4 q = lds_f4(tile + 16u * (j + u));
      if (KIND == KRMU && ACC != kAccCount) wj[u] = __uint_as_float(lds_u32(wtile + 4u * (j + u)));
      else wj[u] = q.w;
      if constexpr ((KIND == KMONO || KIND == KTHETA) && M0 == kArith) {
        const float2 qx = make_float2(q.x, q.x), qy = make_float2(q.y, q.y),
                     qz = make_float2(q.z, q.z);
#pragma unroll
        for (int sp = 0; sp < HP / 2; sp++) {
          uint32_t o[2];
          float2 s2;
          mono_arith2(p.ax[0], qx, qy, qz, h.nx2[sp], h.ny2[sp], h.nz2[sp], st0, c1d, o[0], o[1],
                      s2);
          arith_pair_out<HP, MASK, kLazy>(s2, o, u, sp, gj0 + j + u, h, zoff, thr, off, sc, nmask);
        }
      } else if constexpr ((KIND == KMONO || KIND == KTHETA) &&
                           (M0 == kArithLog || M0 == kArithLogU)) {
        const float2 qx = make_float2(q.x, q.x), qy = make_float2(q.y, q.y),
                     qz = make_float2(q.z, q.z);
#pragma unroll
        for (int sp = 0; sp < HP / 2; sp++) {
          uint32_t o[2];
          float2 s2;
          mono_log2<M0 == kArithLog>(p.ax[0], qx, qy, qz, h.nx2[sp], h.ny2[sp], h.nz2[sp], st0,
                                     c1d, o[0], o[1], s2);
          arith_pair_out<HP, MASK, kLazy>(s2, o, u, sp, gj0 + j + u, h, zoff, thr, off, sc, nmask);
        }
      } else if constexpr (KIND == KSIGPI && M0 == kArith) {
        const float2 qx = make_float2(q.x, q.x), qy = make_float2(q.y, q.y),
                     qz = make_float2(q.z, q.z);
#pragma unroll
        for (int sp = 0; sp < HP / 2; sp++) {
          uint32_t o[2];
          float2 s2;
          sigpi_arith2(p.ax[0], p.ax[1], qx, qy, qz, h.nx2[sp], h.ny2[sp], h.nz2[sp], sl1, st1,
                       c2d, o[0], o[1], s2);
          arith_pair_out<HP, MASK, kLazy>(s2, o, u, sp, gj0 + j + u, h, zoff, thr, off, sc, nmask);
        }
      } else if constexpr (KIND == KRMU && M0 == kArith) {
        const float2 qx = make_float2(q.x, q.x), qy = make_float2(q.y, q.y),
                     qz = make_float2(q.z, q.z);
#pragma unroll
        for (int sp = 0; sp < HP / 2; sp++) {
          uint32_t o[2];
          float2 s2;
          rmu_arith2(p.ax[0], p.ax[1], qx, qy, qz, make_float2(q.w, q.w), h.nx2[sp], h.ny2[sp],
                     h.nz2[sp], h.nq2[sp], h.c2[sp], k2, nk, sl1, st1, c2d, o[0], o[1], s2);
          arith_pair_out<HP, MASK, kLazy>(s2, o, u, sp, gj0 + j + u, h, zoff, thr, off, sc, nmask);
        }
      } else {
        // table binning: the values of two pairs in packed FP32, then a
        // lookup for each
        const float2 qx = make_float2(q.x, q.x), qy = make_float2(q.y, q.y),
                     qz = make_float2(q.z, q.z);
#pragma unroll
        for (int sp = 0; sp < HP / 2; sp++) {
          float2 va, vb;
          if constexpr (KIND == KRMU) {
            const Rmu2 v = rmu_values2(qx, qy, qz, make_float2(q.w, q.w), h.nx2[sp], h.ny2[sp],
                                       h.nz2[sp], h.nq2[sp], h.c2[sp], k2, nk);
            const float2 pl = __fmul2_rn(v.r2, v.l2);
            va = v.r2;
            vb = __fmul2_rn(make_float2(fabsf(v.sl.x), fabsf(v.sl.y)),
                            make_float2(rsqrt_hw(pl.x), rsqrt_hw(pl.y)));
          } else {
            const float2 dx = __fadd2_rn(qx, h.nx2[sp]), dy = __fadd2_rn(qy, h.ny2[sp]),
                         dz = __fadd2_rn(qz, h.nz2[sp]);
            if constexpr (KIND == KSIGPI) {
              va = __ffma2_rn(dy, dy, __fmul2_rn(dx, dx));
              vb = __fmul2_rn(dz, dz);
            } else {
              va = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
              vb = va;
            }
          }
#pragma unroll
          for (int e = 0; e < 2; e++) {
            const int s = 2 * sp + e, k = u * HP + s;
            bool near;
            uint32_t o = table_slot<KIND, M0, M1>(p, lut, band, e ? va.y : va.x,
                                                  e ? vb.y : vb.x, near) + zoff;
            const int gj = gj0 + j + u;
            if (MASK == 1 && !(gj > h.id[s])) { o = zoff; near = false; }  // not a pair of this item
            if (MASK == 2 && gj == h.id[s]) { o = zoff; near = false; }    // no self pair
            if (near) { o = zoff; nmask |= 1u << k; }
            off[k] = o;
          }
        }
      }
    }
    if (ACC != kAccAdjoint) {
#pragma unroll
      for (int k = 0; k < NP; k++) red_add1(kDirect ? off[k] : w.s_hist_lane + off[k]);
    }
    if (ACC == kAccIntWeighted) {
      // the weight product, an exact integer below 2^22: its bits from
      // p + 2^23 (exact), added to the weight histogram (same slot offset)
#pragma unroll
      for (int k = 0; k < NP; k++) {
        const float pw = __fadd_rn(__fmul_rn(h.w[k % HP], wj[k / HP]), 8388608.0f);
        red_add_u32(off[k] + w.s_dw, __float_as_uint(pw) - 0x4B000000u);
      }
    }
    if (ACC == kAccWeighted) {
      // lane-private float-float column: a read-modify-write, no atomics
#pragma unroll
      for (int k = 0; k < NP; k++) {
        const float a = h.w[k % HP], b = wj[k / HP];
        const float ph = __fmul_rn(a, b);
        const float pl = __fmaf_rn(a, b, -ph);  // exact: a * b = ph + pl
        const uint32_t c = w.s_wcol + 8u * (off[k] >> slot_shift);
        float2 v = lds_f2(c);
        ff_add(v.x, v.y, ph, pl);
        sts_f2(c, v);
      }
    }
    if (ACC == kAccAdjoint) {
#pragma unroll
      for (int k = 0; k < NP; k++) {
        const float2 g = lds_f2(w.s_G + 8u * (off[k] >> slot_shift));  // slot 0, trash: 0
        const float b = wj[k / HP];
        const float th = __fmul_rn(b, g.x);
        const float tl = __fmaf_rn(b, g.y, __fmaf_rn(b, g.x, -th));
        ff_add(h.gh[k % HP], h.gl[k % HP], th, tl);
      }
    }
    bool flagged;
    if constexpr (kLazy) {
      // the step's largest score (a tree: short dependency chains)
      float m[NP];
#pragma unroll
      for (int k = 0; k < NP; k++) m[k] = sc[k];
#pragma unroll
      for (int d = 1; d < NP; d *= 2)
#pragma unroll
        for (int k = 0; k + d < NP; k += 2 * d) m[k] = fmaxf(m[k], m[k + d]);
      flagged = __any_sync(kFull, m[0] >= thr);
    } else {
      flagged = __any_sync(kFull, nmask != 0u);
    }
    // rare: pairs inside an edge's error band join the warp's re-test queue;
    // the queue only grows here, so it is drained here when it holds 32.
    // A flagged step usually holds one near pair in the whole warp, and the
    // warp issues whatever any lane needs: so only the step positions k near
    // in some lane are handled (the lanes' near masks OR-ed across the
    // warp), each with its own compile-time k, so off[k] and sc[k] stay
    // in registers.
    if (flagged) {
      // pairs with the padding rows past this item's rows are never queued
      // (a culled run: rows past the end of its real rows; the neighbour
      // index of a queued pair's row is looked up only then)
      const int lim = MASK == 0 ? (int)lds_u32(w.s_box + 28u) : w.gje;
      unsigned lm = 0;  // this lane's near positions
#pragma unroll
      for (int k = 0; k < NP; k++)
        if (kLazy ? (sc[k] >= thr) : ((nmask >> k) & 1u) != 0u) lm |= 1u << k;
      unsigned wm = __reduce_or_sync(kFull, lm);  // the warp's
      auto near_pair = [&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const bool nk = ((lm >> k) & 1u) != 0u;
        if (kLazy && nk) {
          // take back what the FP32 slot received: its count, and the weight
          // product (weighted) or the gradient term (adjoint), by the
          // opposite float-float addition (exact up to the columns' own
          // 2^-48 rounding)
          if (ACC != kAccAdjoint)
            red_add_u32(kDirect ? off[k] : w.s_hist_lane + off[k], 0xffffffffu);
          if (ACC == kAccIntWeighted) {
            const float pw = __fadd_rn(__fmul_rn(h.w[k % HP], wj[k / HP]), 8388608.0f);
            red_add_u32(off[k] + w.s_dw, 0x4B000000u - __float_as_uint(pw));
          }
          if (ACC == kAccWeighted) {
            const float a = h.w[k % HP], b = wj[k / HP];
            const float ph = __fmul_rn(a, b);
            const float pl = __fmaf_rn(a, b, -ph);
            const uint32_t c = w.s_wcol + 8u * (off[k] >> slot_shift);
            float2 v = lds_f2(c);
            ff_add(v.x, v.y, -ph, -pl);
            sts_f2(c, v);
          }
          if (ACC == kAccAdjoint) {
            const float2 gg = lds_f2(w.s_G + 8u * (off[k] >> slot_shift));
            const float b = wj[k / HP];
            const float th = __fmul_rn(b, gg.x);
            const float tl = __fmaf_rn(b, gg.y, __fmaf_rn(b, gg.x, -th));
            ff_add(h.gh[k % HP], h.gl[k % HP], -th, -tl);
          }
        }
        // (a padded home slot or tile row is never a pair, whatever its
        // arithmetic gave)
        const int gjk = gj0 + j + k / HP;
        if (nk && h.id[k % HP] != 0x7fffffff && gjk < lim) {
          near_count++;
          int pos = atomicAdd(w.qcnt, 1);
          if (pos < w.qcap)
            w.queue[pos] = make_int2(
                h.id[k % HP],
                MASK != 0 ? gjk
                          : (int)lds_u32(kIdxRow ? tile + 16u * (uint32_t)(j + k / HP) + 12u
                                                 : w.s_cidx + 4u * gjk));
          else atomicCAS(p.err, 0, (int)CUTE_E_DEVICE);
        }
      };
      static_assert(NP == 8, "eight step positions");
      while (wm) {  // warp-uniform
        const int k = __ffs(wm) - 1;
        wm &= wm - 1u;
        switch (k) {
          case 0: near_pair(std::integral_constant<int, 0>{}); break;
          case 1: near_pair(std::integral_constant<int, 1>{}); break;
          case 2: near_pair(std::integral_constant<int, 2>{}); break;
          case 3: near_pair(std::integral_constant<int, 3>{}); break;
          case 4: near_pair(std::integral_constant<int, 4>{}); break;
          case 5: near_pair(std::integral_constant<int, 5>{}); break;
          case 6: near_pair(std::integral_constant<int, 6>{}); break;
          default: near_pair(std::integral_constant<int, 7>{}); break;
        }
      }
      __syncwarp();
      if (*w.qcnt >= 32) process_queue<KIND, ACC>(p, pd, w, lane, false);
    }
  }
}

template <int KIND, int HP, int M0, int M1, int ACC>
__device__ __forceinline__ void tile_dispatch_mask(const KParams &p, uint32_t lut,
                                                   uint32_t band, const PairDev &pd,
                                                   const WarpSmem &w, uint32_t tile, uint32_t wtile, int cnt,
                                                   int gj0, Home<HP> &h, int lane, int mask,
                                                   unsigned &dc) {
  if (mask == 1) tile_pairs<KIND, HP, M0, M1, 1, ACC>(p, lut, band, pd, w, tile, wtile, cnt, gj0, h, lane, dc);
  else if (ACC == kAccAdjoint && mask == 2)
    tile_pairs<KIND, HP, M0, M1, 2, ACC>(p, lut, band, pd, w, tile, wtile, cnt, gj0, h, lane, dc);
  else tile_pairs<KIND, HP, M0, M1, 0, ACC>(p, lut, band, pd, w, tile, wtile, cnt, gj0, h, lane, dc);
}

template <int KIND, int HP, int ACC>
__device__ __forceinline__ void tile_dispatch(const KParams &p, uint32_t lut,
                                              uint32_t band, const PairDev &pd,
                                              const WarpSmem &w, uint32_t tile, uint32_t wtile, int cnt,
                                              int gj0, Home<HP> &h, int lane, int mask,
                                              unsigned &dc) {
  const int m0 = p.ax[0].mode;
  if (KIND == KMONO || KIND == KTHETA) {
    if (m0 == kArith) tile_dispatch_mask<KIND, HP, kArith, 0, ACC>(p, lut, band, pd, w, tile, wtile, cnt, gj0, h, lane, mask, dc);
    else if (m0 == kArithLog) tile_dispatch_mask<KIND, HP, kArithLog, 0, ACC>(p, lut, band, pd, w, tile, wtile, cnt, gj0, h, lane, mask, dc);
    else if (m0 == kArithLogU) tile_dispatch_mask<KIND, HP, kArithLogU, 0, ACC>(p, lut, band, pd, w, tile, wtile, cnt, gj0, h, lane, mask, dc);
    else if (m0 == kLutLinear) tile_dispatch_mask<KIND, HP, kLutLinear, 0, ACC>(p, lut, band, pd, w, tile, wtile, cnt, gj0, h, lane, mask, dc);
    else tile_dispatch_mask<KIND, HP, kLutLog, 0, ACC>(p, lut, band, pd, w, tile, wtile, cnt, gj0, h, lane, mask, dc);
  } else {
    const int m1 = p.ax[1].mode;
    if (m0 == kArith) {
      tile_dispatch_mask<KIND, HP, kArith, kArith, ACC>(p, lut, band, pd, w, tile, wtile, cnt, gj0, h, lane, mask, dc);
    } else if (m0 == kLutLinear) {
      if (m1 == kLutLinear) tile_dispatch_mask<KIND, HP, kLutLinear, kLutLinear, ACC>(p, lut, band, pd, w, tile, wtile, cnt, gj0, h, lane, mask, dc);
      else tile_dispatch_mask<KIND, HP, kLutLinear, kLutLog, ACC>(p, lut, band, pd, w, tile, wtile, cnt, gj0, h, lane, mask, dc);
    } else {
      if (m1 == kLutLinear) tile_dispatch_mask<KIND, HP, kLutLog, kLutLinear, ACC>(p, lut, band, pd, w, tile, wtile, cnt, gj0, h, lane, mask, dc);
      else tile_dispatch_mask<KIND, HP, kLutLog, kLutLog, ACC>(p, lut, band, pd, w, tile, wtile, cnt, gj0, h, lane, mask, dc);
    }
  }
}

__device__ __forceinline__ float shift_of(int code, float L) {
  return code == 1 ? L : (code == 2 ? -L : 0.0f);
}

// Neighbour cull of two rows at once (packed FP32): row q is kept unless
// its distance from the home box exceeds the reach, the gap on each axis
// being max(lo - q, q - hi, 0); sigma, pi: the x-y gap against sigma's
// reach and the z gap against pi's.  The box comes negated (nlo = -lo,
// nhi = -hi), so q - lo and q - hi are additions: the same roundings as
// lo - q (its exact negation) and q - hi.  p.cull_r2 and p.cull_pi are
// widened on the host past the FP32 frame's rounding and this arithmetic's
// own, so no pair within reach is dropped.
template <int KIND>
__device__ __forceinline__ void cull_keep2(const KParams &p, float4 qa, float4 qb, float4 nlo,
                                           float4 nhi, bool &ka, bool &kb) {
  auto gap = [](float a, float b, float nl, float nh, float2 &g) {
    const float2 q = make_float2(a, b);
    const float2 tl = __fadd2_rn(q, make_float2(nl, nl));  // q - lo
    const float2 th = __fadd2_rn(q, make_float2(nh, nh));  // q - hi
    g = make_float2(fmaxf(fmaxf(-tl.x, th.x), 0.0f), fmaxf(fmaxf(-tl.y, th.y), 0.0f));
  };
  float2 gx, gy, gz;
  gap(qa.x, qb.x, nlo.x, nhi.x, gx);
  gap(qa.y, qb.y, nlo.y, nhi.y, gy);
  gap(qa.z, qb.z, nlo.z, nhi.z, gz);
  if (KIND == KSIGPI) {
    const float2 s2 = __ffma2_rn(gy, gy, __fmul2_rn(gx, gx));
    ka = s2.x <= p.cull_r2 && gz.x <= p.cull_pi;
    kb = s2.y <= p.cull_r2 && gz.y <= p.cull_pi;
  } else {
    const float2 d2 = __ffma2_rn(gz, gz, __ffma2_rn(gy, gy, __fmul2_rn(gx, gx)));
    ka = d2.x <= p.cull_r2;
    kb = d2.y <= p.cull_r2;
  }
}

// One landed tile of a culled item, compacted in place: the rows within
// reach of the home box move to the front of the tile (a ballot and a
// prefix count place them; a tile kept whole stays where it is), right
// behind the rows carried from the tile before into the buffer's kTilePre
// leading rows.  Sets the run to pair -- rows [base, base + m), whole steps
// (the item's last tile pads to a step with sentinel rows) -- and leaves in
// the box words the rows short of a step and where they start, for
// cull_carry.  Nothing of this lives in registers across the pairing.
// cand gains this lane's evaluated pairs, slots the pair slots run.
template <int KIND, int HP, int ACC>
__device__ __forceinline__ void cull_compact(const KParams &p, const WarpSmem &w, int tt, int js,
                                             int je, bool last, const Home<HP> &h, int lane,
                                             unsigned long long &cand, unsigned long long &slots,
                                             int &base, int &m) {
  constexpr bool kWTile = KIND == KRMU && ACC != kAccCount;
  constexpr bool kIdxRow = ACC == kAccCount && KIND != KRMU;
  constexpr int U = 8 / HP;  // rows per step of tile_pairs
  static_assert(kTile == 64, "two rows per lane");
  static_assert(U - 1 <= kTilePre && U - 1 <= kTileRows - kTilePre - kTile,
                "carry and padding room");
  const uint32_t B = smem_addr(w.tiles + (tt & 1) * kTileRows);
  const uint32_t WB = smem_addr(w.wtiles + (tt & 1) * kTileRows);
  const int g0 = js + tt * kTile;
  const uint32_t ra = (uint32_t)(kTilePre + lane), rb = ra + 32u;  // this lane's rows
  const float4 qa = lds_f4(B + 16u * ra), qb = lds_f4(B + 16u * rb);
  const float4 nlo = lds_f4(w.s_box), nhi = lds_f4(w.s_box + 16u);
  const int nbuf = __float_as_int(nlo.w);  // rows carried in
  bool ka, kb;
  cull_keep2<KIND>(p, qa, qb, nlo, nhi, ka, kb);
  const unsigned ba = __ballot_sync(kFull, ka && g0 + lane < je);
  const unsigned bb = __ballot_sync(kFull, kb && g0 + lane + 32 < je);
  int kept;
  if ((ba & bb) == kFull) {  // every row kept: in place already
    sts_u32(kIdxRow ? B + 16u * ra + 12u : w.s_cidx + 4u * ra, (uint32_t)(g0 + lane));
    sts_u32(kIdxRow ? B + 16u * rb + 12u : w.s_cidx + 4u * rb, (uint32_t)(g0 + lane + 32));
    kept = kTile;
  } else {
    const float wa = kWTile ? __uint_as_float(lds_u32(WB + 4u * ra)) : 0.0f;
    const float wb = kWTile ? __uint_as_float(lds_u32(WB + 4u * rb)) : 0.0f;
    const unsigned below = (1u << lane) - 1u;
    const int na = __popc(ba);
    __syncwarp();  // every row read before any moves
    if ((ba >> lane) & 1u) {
      const uint32_t r = (uint32_t)(kTilePre + __popc(ba & below));
      const int gi = g0 + lane;
      sts_f4(B + 16u * r, kIdxRow ? make_float4(qa.x, qa.y, qa.z, __int_as_float(gi)) : qa);
      if (!kIdxRow) sts_u32(w.s_cidx + 4u * r, (uint32_t)gi);
      if (kWTile) sts_u32(WB + 4u * r, __float_as_uint(wa));
    }
    if ((bb >> lane) & 1u) {
      const uint32_t r = (uint32_t)(kTilePre + na + __popc(bb & below));
      const int gi = g0 + lane + 32;
      sts_f4(B + 16u * r, kIdxRow ? make_float4(qb.x, qb.y, qb.z, __int_as_float(gi)) : qb);
      if (!kIdxRow) sts_u32(w.s_cidx + 4u * r, (uint32_t)gi);
      if (kWTile) sts_u32(WB + 4u * r, __float_as_uint(wb));
    }
    kept = na + __popc(bb);
  }
  int nv = 0;  // this lane's occupied home slots: its evaluated pairs
#pragma unroll
  for (int s = 0; s < HP; s++) nv += h.id[s] != 0x7fffffff;
  cand += (unsigned)(kept * nv);
  base = kTilePre - nbuf;
  const int n = nbuf + kept;  // the run: rows [base, base + n)
  m = last ? (n + U - 1) & ~(U - 1) : n & ~(U - 1);
  slots += (unsigned)(32 * HP * m);
  if (last && lane < m - n) {  // (never queued: past the real rows)
    const uint32_t r = (uint32_t)(base + n + lane);
    sts_f4(B + 16u * r, make_float4(-p.far, -p.far, -p.far, 0.0f));
    if (kWTile) sts_u32(WB + 4u * r, 0u);
  }
  if (lane == 0) {  // the rows short of a step (for cull_carry), the end of the real rows
    sts_u32(w.s_box + 12u, (uint32_t)(last ? 0 : n - m));
    sts_u32(w.s_box + 28u, (uint32_t)(base + n));
  }
  __syncwarp();
}

// After the run of tile tt is paired: its rows short of a step move to the
// other buffer's rows [kTilePre - rem, kTilePre), which the cp.async of the
// next tile does not write; their indices may overlap the targets in
// s_cidx, so every lane reads before any lane writes.  rem becomes the
// next tile's carried-in count.
template <int KIND, int ACC>
__device__ __forceinline__ void cull_carry(const WarpSmem &w, int tt, int lane) {
  constexpr bool kWTile = KIND == KRMU && ACC != kAccCount;
  constexpr bool kIdxRow = ACC == kAccCount && KIND != KRMU;
  __syncwarp();
  const int rem = (int)lds_u32(w.s_box + 12u);
  if (rem == 0) return;
  const uint32_t f = lds_u32(w.s_box + 28u) - (uint32_t)rem + (uint32_t)lane;
  const uint32_t B = smem_addr(w.tiles + (tt & 1) * kTileRows);
  const uint32_t WB = smem_addr(w.wtiles + (tt & 1) * kTileRows);
  float4 cq = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  uint32_t ci = 0u, cw = 0u;
  if (lane < rem) {
    cq = lds_f4(B + 16u * f);
    if (!kIdxRow) ci = lds_u32(w.s_cidx + 4u * f);
    if (kWTile) cw = lds_u32(WB + 4u * f);
  }
  __syncwarp();
  if (lane < rem) {
    const uint32_t t = (uint32_t)(kTilePre - rem + lane);
    sts_f4(smem_addr(w.tiles + ((tt + 1) & 1) * kTileRows) + 16u * t, cq);
    if (!kIdxRow) sts_u32(w.s_cidx + 4u * t, ci);
    if (kWTile) sts_u32(smem_addr(w.wtiles + ((tt + 1) & 1) * kTileRows) + 4u * t, cw);
  }
}

template <int KIND, bool PER, int HP, int ACC>
__global__ void __launch_bounds__(32 * count_max_warps(KIND == KMONO, HP, ACC), 1)
    k_count(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr bool kWTile = KIND == KRMU && ACC != kAccCount;
  constexpr bool kIdxRow = ACC == kAccCount && KIND != KRMU;  // culled rows' index: weight word
  const SmemLayout L = smem_layout(p.lut_words, p.band_words, p.nslots, p.R, HP, ACC, kWTile,
                                   !kIdxRow);
  uint32_t *lut = (uint32_t *)smem;
  for (int i = threadIdx.x; i < p.lut_words; i += blockDim.x) lut[i] = p.lut[i];
  float2 *band = (float2 *)(smem + align16(p.lut_words * 4));
  for (int i = threadIdx.x; i < p.band_words; i += blockDim.x) band[i] = p.band[i];
  float2 *Gs = (float2 *)(smem + align16(p.lut_words * 4) + align16(p.band_words * 8));
  if (ACC == kAccAdjoint) {
    // G per slot as float-float; slot 0 and the out-of-range slots hold 0
    for (int s = threadIdx.x; s < p.nslots; s += blockDim.x) {
      int s0 = s / p.slots1, s1 = s - s0 * p.slots1;
      bool in = s0 >= 1 && s0 <= p.n0 && (p.slots1 == 1 || (s1 >= 1 && s1 <= p.n1));
      double g = in ? p.G[(s0 - 1) * p.n1 + (p.slots1 == 1 ? 0 : s1 - 1)] : 0.0;
      float gh = (float)g;
      Gs[s] = make_float2(gh, (float)(g - (double)gh));
    }
  }
  unsigned char *wb = smem + L.lut_bytes + (size_t)warp * L.warp_bytes;
  WarpSmem w;
  w.hist = (uint32_t *)wb;
  w.s_dw = (uint32_t)align16(p.nslots * p.R * 4);
  w.whist = (uint32_t *)(wb + w.s_dw);
  w.hist_lane = (char *)wb + (lane & (p.R - 1)) * 4;
  w.wstride = p.nslots + 1;  // odd stride: the flush reads across columns conflict-free
  w.wall = (float2 *)(wb + align16(p.nslots * p.R * 4));
  w.wcol = w.wall + lane * w.wstride;
  w.G = Gs;
  w.qcnt = (int *)(wb + L.hist_bytes);
  w.queue = (int2 *)(wb + L.hist_bytes + 16);
  w.qcap = L.queue_cap;
  w.tiles = (float4 *)(wb + L.hist_bytes + L.queue_bytes);
  w.wtiles = (float *)(wb + L.hist_bytes + L.queue_bytes + L.tile_bytes);
  w.s_box = smem_addr(wb + L.hist_bytes + L.queue_bytes + L.tile_bytes + L.wtile_bytes);
  w.s_cidx = w.s_box + 32u;
  w.s_hist_lane = smem_addr(w.hist_lane);
  w.s_wcol = smem_addr(w.wcol);
  w.s_G = smem_addr(w.G);
  const uint32_t s_lut = smem_addr(lut), s_band = smem_addr(band);
  for (int i = lane; i < p.nslots * p.R; i += 32) w.hist[i] = 0u;
  if (ACC == kAccIntWeighted)
    for (int i = lane; i < p.nslots * p.R; i += 32) w.whist[i] = 0u;
  if (ACC == kAccWeighted)
    for (int i = lane; i < 32 * w.wstride; i += 32) w.wall[i] = make_float2(0.0f, 0.0f);
  if (lane == 0) *w.qcnt = 0;
  __syncthreads();

  int cur_pair = -1;
  PairDev pd;
  unsigned long long acc = 0, accw = 0, items = 0, slots = 0, cand = 0;
  unsigned near_count = 0;
  // Work items in a two-deep pipeline: while an item runs, the record of
  // the next one is in flight and the ticket of the one after it has been
  // drawn (lane 0 holds it until it is needed).
  const int4 rec_none = make_int4(0, 0, 0, 0);
  unsigned long long tk = (lane == 0) ? atomicAdd(p.ticket, 1ull) : 0ull;
  long long it = (long long)__shfl_sync(kFull, tk, 0);
  int4 rec_next = it < p.total ? p.items[it * p.item_stride] : rec_none;
  tk = (lane == 0 && it < p.total) ? atomicAdd(p.ticket, 1ull) : 0ull;
  for (;;) {
    if (it >= p.total) break;
    const int4 rec = rec_next;
    it = (long long)__shfl_sync(kFull, tk, 0);
    rec_next = it < p.total ? p.items[it * p.item_stride] : rec_none;
    tk = (lane == 0 && it < p.total) ? atomicAdd(p.ticket, 1ull) : 0ull;
    const int pi = (int)((unsigned)rec.w >> 16);
    if (pi != cur_pair) {
      if (cur_pair >= 0) {
        process_queue<KIND, ACC>(p, pd, w, lane, true);
        if (ACC != kAccAdjoint) flush_hist(p, w, pd.out, lane);
        if (ACC == kAccIntWeighted) flush_whist(p, w, pd.out, lane);
        acc = accw = 0;
      }
      cur_pair = pi;
      pd = p.pairs[cur_pair];
    }
    const int hs = rec.x, he = hs + (rec.w & 0xff), js = rec.y, je = rec.z;
    const int mask = (rec.w >> 8) & 3;
    if (mask == 1 && je <= hs + 1) continue;  // every j precedes every i
    // uint32 overflow guard: increments a copy can receive from this item
    if (ACC != kAccAdjoint) {
      const unsigned long long bound = 2ull * (32 / p.R) * HP * (unsigned long long)(je - js);
      // (integer weights: each increment of the weight histogram is at most
      // the largest product; the host keeps one item's total below 2^32)
      const unsigned long long bw = ACC == kAccIntWeighted ? bound * p.wpmax : 0ull;
      if (acc + bound > 0xFFFFFFFFull || accw + bw > 0xFFFFFFFFull) {
        process_queue<KIND, ACC>(p, pd, w, lane, true);
        flush_hist(p, w, pd.out, lane);
        if (ACC == kAccIntWeighted) flush_whist(p, w, pd.out, lane);
        acc = accw = 0;
      }
      acc += bound;
      accw += bw;
    }
    items++;
    // Rows of other cells (and every row of a cross count) go through the
    // neighbour cull; the home run against its own cells does not.
    const bool cull = !(mask == 1 || (ACC == kAccAdjoint && mask == 2));
    if (!cull)
      slots += (unsigned long long)(32 * HP) * (unsigned long long)((je - js + (8 / HP) - 1) & ~((8 / HP) - 1));

    // the first tile is in flight while the home objects load
    const int nj = je - js;
    const int ntiles = (nj + kTile - 1) / kTile;
    // R_MU tiles come from (x, y, z, q), and their weights from (x, y, z, w)
    const float4 *srcB = KIND == KRMU ? pd.qB : pd.posB;
    auto load_tile = [&](int tt) {
      float4 *dst = w.tiles + (tt & 1) * kTileRows + kTilePre;
      float *wdst = w.wtiles + (tt & 1) * kTileRows + kTilePre;
      for (int e = lane; e < kTile; e += 32) {
        const int g = js + tt * kTile + e;
        if (g < je) {
          cp_async16(dst + e, srcB + g);
          if (kWTile) cp_async4(wdst + e, &pd.posB[g].w);
        } else {
          dst[e] = make_float4(-p.far, -p.far, -p.far, 0.0f);
          if (kWTile) wdst[e] = 0.0f;
        }
      }
      cp_async_commit();
    };
    load_tile(0);
    const int code = (rec.w >> 10) & 63;
    const float Sx = PER ? shift_of(code & 3, pd.L32) : 0.0f;
    const float Sy = PER ? shift_of((code >> 2) & 3, pd.L32) : 0.0f;
    const float Sz = PER ? shift_of((code >> 4) & 3, pd.L32) : 0.0f;
    Home<HP> h;
#pragma unroll
    for (int s = 0; s < HP; s++) {
      const int idx = hs + lane + 32 * s;
      h.gh[s] = 0.0f;
      h.gl[s] = 0.0f;
      if (idx < he) {
        const float4 a = KIND == KRMU ? pd.qA[idx] : pd.posA[idx];
        Home<HP>::put(h.nx2, s, -__fsub_rn(a.x, Sx));
        Home<HP>::put(h.ny2, s, -__fsub_rn(a.y, Sy));
        Home<HP>::put(h.nz2, s, -__fsub_rn(a.z, Sz));
        h.w[s] = KIND == KRMU ? (ACC == kAccWeighted ? pd.posA[idx].w : 1.0f) : a.w;
        h.id[s] = idx;
        // candidate pairs of the rows not culled: j in [js, je), with j > i
        // (self) or j != i
        if (!cull)
          cand += mask == 1 ? (unsigned)max(0, je - max(js, idx + 1))
                            : (unsigned)(nj - (mask == 2 && idx >= js && idx < je ? 1 : 0));
        if (KIND == KRMU) {
          // C_i = k (2 q_i + 4 q0), rounded once from FP64
          Home<HP>::put(h.nq2, s, -a.w);
          Home<HP>::put(h.c2, s, (float)((double)p.ax[1].lsc *
                                         __dadd_rn(__dmul_rn(2.0, (double)a.w), __dmul_rn(4.0, pd.q0))));
        }
      } else {
        Home<HP>::put(h.nx2, s, -p.far);
        Home<HP>::put(h.ny2, s, -p.far);
        Home<HP>::put(h.nz2, s, -p.far);
        h.w[s] = 0.0f;
        h.id[s] = 0x7fffffff;
        if (KIND == KRMU) {  // k l.l < 0: mu is NaN and clamps to the top slot
          Home<HP>::put(h.nq2, s, 0.0f);
          Home<HP>::put(h.c2, s, 0.0f);
        }
      }
    }
    w.gje = je;
    if (cull) {
      // bounding box of the home objects in the image frame (x_i - shift),
      // kept in shared memory beside the culled rows
      float bl[3] = {3.0e38f, 3.0e38f, 3.0e38f}, bh[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
#pragma unroll
      for (int s = 0; s < HP; s++) {
        if (h.id[s] != 0x7fffffff) {
          const float c[3] = {-Home<HP>::get(h.nx2, s), -Home<HP>::get(h.ny2, s),
                              -Home<HP>::get(h.nz2, s)};
#pragma unroll
          for (int k = 0; k < 3; k++) {
            bl[k] = fminf(bl[k], c[k]);
            bh[k] = fmaxf(bh[k], c[k]);
          }
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 3; k++) {
          bl[k] = fminf(bl[k], __shfl_xor_sync(kFull, bl[k], o));
          bh[k] = fmaxf(bh[k], __shfl_xor_sync(kFull, bh[k], o));
        }
      if (lane == 0) {  // negated: (-lo, carried rows 0), (-hi, -)
        sts_f4(w.s_box, make_float4(-bl[0], -bl[1], -bl[2], 0.0f));
        sts_f4(w.s_box + 16u, make_float4(-bh[0], -bh[1], -bh[2], 0.0f));
      }
    }

    for (int tt = 0; tt < ntiles; tt++) {
      if (tt + 1 < ntiles) {
        load_tile(tt + 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
      // the run to pair: the landed tile, or its culled rows (one dispatch
      // for both, so the pairing loop is compiled once per mask)
      const uint32_t B = smem_addr(w.tiles + (tt & 1) * kTileRows);
      const uint32_t WB = smem_addr(w.wtiles + (tt & 1) * kTileRows);
      int first = kTilePre, cnt, gj0 = js + tt * kTile;
      if (!cull) {
        cnt = min(kTile, nj - tt * kTile);
        cnt = (cnt + (8 / HP) - 1) & ~((8 / HP) - 1);  // whole steps; padded rows are sentinels
      } else {
        cull_compact<KIND, HP, ACC>(p, w, tt, js, je, tt + 1 == ntiles, h, lane, cand, slots,
                                    first, cnt);
        gj0 = first;  // (culled rows: their indices are in s_cidx)
      }
      if (cnt > 0)
        tile_dispatch<KIND, HP, ACC>(p, s_lut, s_band, pd, w, B + 16u * first, WB + 4u * first,
                                     cnt, gj0, h, lane, cull ? 0 : mask, near_count);
      if (cull && tt + 1 < ntiles) cull_carry<KIND, ACC>(w, tt, lane);
      __syncwarp();
    }
    if (ACC == kAccWeighted) flush_wsum(p, w, pd.out, lane);
    if (ACC == kAccAdjoint) {
#pragma unroll
      for (int s = 0; s < HP; s++) {
        const int idx = hs + lane + 32 * s;
        const double g = (double)h.gh[s] + (double)h.gl[s];
        if (idx < he && g != 0.0) atomicAdd(&p.grad[pd.permA[idx]], g);
      }
    }
  }
  if (cur_pair >= 0) {
    process_queue<KIND, ACC>(p, pd, w, lane, true);
    if (ACC != kAccAdjoint) flush_hist(p, w, pd.out, lane);
    if (ACC == kAccIntWeighted) flush_whist(p, w, pd.out, lane);
  }
  if (lane == 0 && items) atomicAdd(&p.stats[1], items);
  if (lane == 0 && slots) atomicAdd(&p.stats[3], slots);
  for (int o = 16; o > 0; o >>= 1) cand += __shfl_xor_sync(kFull, cand, o);
  if (lane == 0 && cand) atomicAdd(&p.stats[4], cand);
  for (int o = 16; o > 0; o >>= 1) near_count += __shfl_xor_sync(kFull, near_count, o);
  if (lane == 0 && near_count) atomicAdd(&p.stats[2], (unsigned long long)near_count);
}

template <int KIND, bool PER, int HP, int ACC>
cudaError_t launch_count_t(const KParams &p, int blocks, int threads, size_t smem, cudaStream_t st) {
  auto fn = k_count<KIND, PER, HP, ACC>;
  // the shared-memory opt-in is a host call of a few microseconds: made once
  // per instantiation and device, for the device's whole opt-in limit
  static std::atomic<int> opted[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices || !opted[dev].load()) {
    int lim = 0;
    e = cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             std::max(lim, (int)smem));
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDevices) opted[dev].store(1);
  }
  fn<<<blocks, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <int KIND, bool PER, int ACC>
cudaError_t launch_count_hp(const KParams &p, int hp, int blocks, int threads, size_t smem,
                            cudaStream_t st) {
  if (hp == 2) return launch_count_t<KIND, PER, 2, ACC>(p, blocks, threads, smem, st);
  return launch_count_t<KIND, PER, 4, ACC>(p, blocks, threads, smem, st);
}

template <int KIND, bool PER>
cudaError_t launch_count_acc(const KParams &p, int acc, int hp, int blocks, int threads,
                             size_t smem, cudaStream_t st) {
  if constexpr (KIND == KMONO) {
    if (acc == kAccIntWeighted)
      return launch_count_hp<KIND, PER, kAccIntWeighted>(p, hp, blocks, threads, smem, st);
  }
  if (acc == kAccWeighted) return launch_count_hp<KIND, PER, kAccWeighted>(p, hp, blocks, threads, smem, st);
  if (acc == kAccAdjoint) return launch_count_hp<KIND, PER, kAccAdjoint>(p, hp, blocks, threads, smem, st);
  return launch_count_hp<KIND, PER, kAccCount>(p, hp, blocks, threads, smem, st);
}

}  // namespace cute

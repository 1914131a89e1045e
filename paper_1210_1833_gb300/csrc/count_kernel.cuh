// count_kernel.cuh -- the pair-counting kernel (Sec. 3.1-3.2: distance, bin,
// histogram increment for every candidate pair; Sec. 3.3: candidates from
// neighbouring cells only).
//
// Design on sm_103a (one persistent CTA per SM, warps independent):
//   * work items: (home chunk of catalog A, neighbour slice of catalog B),
//     handed out by a global ticket; each warp holds 32 x HP home objects in
//     registers (HP per lane) and streams the slice through a per-warp
//     double-buffered shared-memory tile filled with cp.async (16-byte,
//     coalesced float4 rows); every lane reads each neighbour as a
//     broadcast and pairs it with its HP home objects;
//   * FP32 separations; the squared separation (and mu) is looked up in a
//     shared-memory table whose clean cells give the byte offset of the
//     histogram slot directly;
//   * per-warp shared-memory histograms, R copies interleaved so lane l
//     increments copy l % R (conflict-free when R = 32), uint32 counters
//     flushed to uint64 in HBM before they could overflow;
//   * pairs in a dirty cell are refined against the one edge's FP32 band,
//     and pairs inside the band go to a per-warp queue that the warp
//     re-tests 32 at a time: a double-float stage with a carried error
//     bound (df_stage.h), the canonical FP64 formulas for what it leaves
//     open.
#pragma once

#include "cute_internal.h"
#include "df_stage.h"

namespace cute {

constexpr int kTile = 64;          // neighbour objects per shared-memory tile
// A tile buffer holds kTilePre rows before the tile (culled rows carried
// from the tile before: fewer than a step, at most 3) and room after it to
// pad the last step.
constexpr int kTilePre = 3;
constexpr int kTileRows = kTilePre + kTile + 3;
constexpr unsigned kFull = 0xffffffffu;

// FP32 sentinels for padded home slots (+far on every axis) and tile rows
// (-far), far = KParams::far: far from everything and from each other, so
// every pair involving one is out of range.  The default far = 1e9: the grid
// frame holds |x| <= 1e8 (checked when the grid is built; image shifts of a
// periodic box add at most 2e8), so every pair with a sentinel is more than
// 5e8 apart, beyond any reach, with squared separations and (r, mu) products
// that stay finite in FP32 ((r, mu) padded home slots give a NaN mu, which
// the top clamp turns into the top slot).  Chord counts binned by kArithLogU
// take far = 1.25 (frame half-extent + reach) instead, the planner's bound on
// the values their spare slots must hold.

// ------------------------------------------------------------------ work entries
// One contiguous range [j0, j1) of catalog B that a home chunk meets, with
// its flags (kSegSelf / kSegNoSelfPair, image shift code in bits 8..13).
struct Seg {
  int j0, j1, flags;
};

// Segments of work entry (chunk c, stencil row r) of pair set pd, in a fixed
// order; returns their number (0..3).  cs is catalog B's cell_start (device
// or host copy).  Every pair of objects within reach is met by exactly one
// entry: cross counts and full stencils pair each chunk with the whole
// x-range of every stencil row; the half stencil of an auto count pairs a
// chunk with its own cell run (j > i) and the cells after it on the home row,
// and with the later rows in full.
__host__ __device__ inline int entry_segments(const PairWork &pd, const int32_t *cs, int4 c, int4 r,
                                              Seg s[3]) {
  const int nx = pd.nx, ny = pd.ny, nz = pd.nz;
  const bool per = pd.periodic != 0;
  const int cx0 = c.z & 0xffff, cx1 = c.z >> 16, cy = c.w & 0xffff, cz = c.w >> 16;
  int y = cy + r.x, z = cz + r.y, sy = 0, sz = 0;
  if (per) {
    if (y < 0) { y += ny; sy = 2; } else if (y >= ny) { y -= ny; sy = 1; }
    if (z < 0) { z += nz; sz = 2; } else if (z >= nz) { z -= nz; sz = 1; }
  } else if (y < 0 || y >= ny || z < 0 || z >= nz) {
    return 0;
  }
  const int32_t *row = cs + ((size_t)z * ny + y) * nx;
  const int syz = (sy << 2) | (sz << 4);
  int n = 0, xa, xb, f;
  if (r.w && pd.mode == kModeAutoHalf) {
    // A and B are one catalog: the chunk against the rest of its cell run
    const int e = row[cx1 + 1];
    if (e > c.x) s[n++] = Seg{c.x, e, kSegSelf};
    xa = cx1 + 1;
    xb = cx1 + r.z;
    f = 0;
  } else {
    xa = cx0 - r.z;
    xb = cx1 + r.z;
    f = (r.w && pd.mode == kModeAutoFull) ? kSegNoSelfPair : 0;
  }
  const int lo = xa > 0 ? xa : 0, hi = xb < nx - 1 ? xb : nx - 1;
  if (per) {
    // the range is never longer than nx: at most the part left of the box
    // (image x - L), the part inside, the part right of it (image x + L)
    if (xa < 0) {
      const int j0 = row[xa + nx], j1 = row[(xb + nx < nx - 1 ? xb + nx : nx - 1) + 1];
      if (j1 > j0) s[n++] = Seg{j0, j1, f | ((2 | syz) << 8)};
    }
    if (lo <= hi) {
      const int j0 = row[lo], j1 = row[hi + 1];
      if (j1 > j0) s[n++] = Seg{j0, j1, f | (syz << 8)};
    }
    if (xb >= nx && n < 3) {
      const int j0 = row[xa - nx > 0 ? xa - nx : 0], j1 = row[xb - nx + 1];
      if (j1 > j0) s[n++] = Seg{j0, j1, f | ((1 | syz) << 8)};
    }
  } else if (lo <= hi) {
    const int j0 = row[lo], j1 = row[hi + 1];
    if (j1 > j0) s[n++] = Seg{j0, j1, f};
  }
  return n;
}

// Work item record (int4): home objects [x, x + (w & 0xff)) of pair set
// w >> 16 against neighbours [y, z); bits 8..9 of w: kSegSelf /
// kSegNoSelfPair, bits 10..15: image shift code.
__host__ __device__ inline int4 item_record(int hs, int he, const Seg &g, int js, int je,
                                            int pair) {
  return make_int4(hs, js, je,
                   (he - hs) | ((g.flags & 3) << 8) | (((g.flags >> 8) & 63) << 10) |
                       (int)((unsigned)pair << 16));
}

// Locate entry e: its pair set (largest p with ebase[p] <= e).
__device__ __forceinline__ int pair_of_entry(const int *__restrict__ ebase, int npairs, int e) {
  int lo = 0, hi = npairs;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (ebase[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

struct SmemLayout {
  int lut_bytes;      // table block: lookup tables, then bands (16-byte multiple)
  int hist_bytes;     // per warp
  int queue_cap;      // per warp entries
  int queue_bytes;
  int tile_bytes;     // per warp (2 tiles)
  int wtile_bytes;    // per warp (2 weight tiles: R_MU weighted / adjoint)
  int cull_bytes;     // per warp: the home box, the culled rows' neighbour indices
                      // (plain counts but (r, mu): in the rows' weight words)
  int warp_bytes;     // per warp total
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

__host__ __device__ inline SmemLayout smem_layout(int lut_words, int band_words, int nslots, int R,
                                                  int HP, int acc, bool wtile, bool idx_array) {
  SmemLayout s;
  // block-wide: lookup tables, bands, and (adjoint) G per slot
  s.lut_bytes = align16(lut_words * 4) + align16(band_words * 8) + (acc == 2 ? align16(nslots * 8) : 0);
  // per warp: the count histogram, and (weighted) 32 float-float columns or
  // (integer weights) a second histogram of the weight products
  s.hist_bytes = align16(nslots * R * 4) + (acc == 1 ? align16(32 * (nslots + 1) * 8) : 0) +
                 (acc == 3 ? align16(nslots * R * 4) : 0);
  s.queue_cap = 32 + 32 * 8;  // checked after every step of 8 pairs per lane
  s.queue_bytes = 16 + align16(s.queue_cap * 8);  // 16-byte header holds the count
  s.tile_bytes = 2 * kTileRows * 16;
  s.wtile_bytes = wtile ? 2 * kTileRows * 4 : 0;
  s.cull_bytes = align16(32 + (idx_array ? kTileRows * 4 : 0));
  // every region, and so every warp's block, starts on a 16-byte boundary
  // (cp.async and float4 rows)
  s.warp_bytes = align16(s.hist_bytes + s.queue_bytes + s.tile_bytes + s.wtile_bytes +
                         s.cull_bytes);
  return s;
}

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared-memory accesses of the hot loop on 32-bit shared-space addresses
// (explicit state space: no generic-address resolution per access).
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ float4 lds_f4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ float2 lds_f2(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts_f2(uint32_t a, float2 v) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void sts_f4(uint32_t a, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}
__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;\n" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void red_add1(uint32_t a) {
  asm volatile("red.shared.add.u32 [%0], 1;\n" ::"r"(a) : "memory");
}
__device__ __forceinline__ void red_add_u32(uint32_t a, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;\n" ::"r"(a), "r"(v) : "memory");
}

// table lookup; MODE fixed per instantiation of the inner loop.  v is
// clamped to the table's range in place (NaN becomes vmax).
template <int MODE>
__device__ __forceinline__ uint32_t lut_get(uint32_t lut, const AxisPlan &a, float &v) {
  v = fminf(v, a.vmax);
  unsigned idx;
  if (MODE == kLutLinear) {
    float t = __fmaf_rn(v, a.scale, 8388608.0f);
    idx = __float_as_uint(t) - 0x4B000000u;
  } else {
    int i = (int)(__float_as_uint(v) >> a.shift) - a.base;
    idx = (unsigned)max(i, 0);
  }
  return lds_u32(lut + 4u * (a.lut_off + idx));
}

// Slot byte offset of value v on an axis whose bands are (lo, hi) pairs;
// near is set when v lies inside the error band of the cell's edge.
__device__ __forceinline__ uint32_t axis_resolve(uint32_t band, const AxisPlan &a, float v,
                                                 uint32_t e, uint32_t stride, bool &near) {
  const uint32_t b = e >> kBandShift;
  uint32_t off = e & kOffMask;
  float2 bd = make_float2(__int_as_float(0x7f800000), __int_as_float(0x7f800000));
  if (b != 0u) bd = lds_f2(band + 8u * (a.band_off + b));
  const bool above = v > bd.y;
  near = (v >= bd.x) && !above;
  return above ? off + stride : off;
}

constexpr float kVFloor = 1e-30f;            // floor of squared separations (finite 1/r)
constexpr float kMagic = 12582912.0f;        // 1.5 * 2^23
constexpr uint32_t kMagicBits = 0x4B400000u;
// 1/sqrt(x) by the hardware approximation (PTX rsqrt.approx.ftz.f32), the
// one rsqrtf() uses for normal inputs; rsqrtf() adds a rescaling for
// subnormal ones, which never occur here (squared separations of FP32
// coordinates are 0 or far above the subnormal range, and the guarded
// operands carry a 1e-30 floor).  The error bounds use rsqrtf's documented
// 2 ulp.
__device__ __forceinline__ float rsqrt_hw(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Uniform edges from 0 (kArith): t = x * inv + cst >= -1/2 for x >= 0 (the
// squared separations carry the kVFloor floor, so x and mu are finite),
// clamped from above to thi (pairs beyond the last edge, padded slots, and
// any non-finite mu);
// tm = t + kMagic holds rint(t) in its low mantissa bits, so the slot
// (bin + 1) is bits(tm) - kMagicBits + 1, and h = t - (tm - kMagic) is exact.
// mono_arith2 / sigpi_arith2 / rmu_arith2 (count_impl.cuh) apply this to two
// pairs at once.

// The same for mu: the band holds the edge, the bound comes from the r slot.
__device__ __forceinline__ uint32_t mu_resolve(uint32_t band, const AxisPlan &a, float mu,
                                               uint32_t e, uint32_t stride, float eps, bool &near) {
  const uint32_t b = e >> kBandShift;
  uint32_t off = e & kOffMask;
  float m = __int_as_float(0x7f800000);
  if (b != 0u) m = lds_f2(band + 8u * (a.band_off + b)).x;
  const float d = __fsub_rn(mu, m);
  near = fabsf(d) <= eps;
  return (d > eps) ? off + stride : off;
}

// ---- canonical FP64 formulas (identical arithmetic to the definition; no
// contraction: every operation is an explicitly rounded intrinsic).  FP64
// runs at a small fraction of the FP32 rate here, so the re-test spends
// FP64 operations only on the canonical values and their edge comparisons.
//
// Minimum image.  The test |d| > L/2 compares the high words (integer
// order of non-negative doubles), which differs from the FP64 test only
// when |d| is within 2^-20 of L/2 -- a separation beyond every reach
// (reach <= 0.47 L), out of range whichever image is taken.
// hi_half: high word of L/2 (periodic), negative for open boundaries.
__device__ __forceinline__ double wrap64(double d, double L, int hi_half) {
  if (hi_half >= 0) {
    const int hi = __double2hiint(d);
    if ((hi & 0x7fffffff) > hi_half) d = (hi < 0) ? __dadd_rn(d, L) : __dsub_rn(d, L);
  }
  return d;
}

// FP32 value of a non-negative double from its high word (relative error
// below 2^-20; 0 below the FP32 normal range, FLT_MAX above it).
__device__ __forceinline__ float approx_f32(double v) {
  const int hi = __double2hiint(v);
  const int e = ((hi >> 20) & 0x7ff) - 1023 + 127;
  if (e <= 0) return 0.0f;
  if (e >= 255) return __int_as_float(0x7f7fffff);
  return __int_as_float((e << 23) | ((hi & 0xfffff) << 3));
}

// Uniform edges from 0: the edge nearest sqrt(v) (v a squared separation),
// in [0, n].  The canonical bin is k or k - 1: the estimate is far closer
// to sqrt(v) than half a bin.
__device__ __forceinline__ int arith_edge(float x, float inv, int n) {
  const int k = __float2int_rn(x * inv);  // NaN gives 0, overflow saturates
  return min(max(k, 0), n);
}
__device__ __forceinline__ float approx_sqrt(double v) {
  const float f = approx_f32(v);
  return f * rsqrt_hw(fmaxf(f, 1e-30f));
}
// bin b with E[b] <= v < E[b+1]; -1 outside
__device__ __forceinline__ int bin64(const double *E, int n, double v) {
  if (!(v >= E[0]) || !(v < E[n])) return -1;
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (v >= E[mid]) lo = mid; else hi = mid;
  }
  return lo;
}
// largest k in [0, n-1] with q >= M[k] * den
__device__ __forceinline__ int mubin64(const double *M, int n, double q, double den) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (q >= __dmul_rn(M[mid], den)) lo = mid; else hi = mid;
  }
  return lo;
}

// bin of a squared separation on axis a (edges E, n bins): one comparison
// with uniform edges, the binary search otherwise; -1 outside
__device__ __forceinline__ int axis_bin64(const AxisPlan &a, const double *E, int n, double v) {
  if (a.mode != kArith) return bin64(E, n, v);
  const int k = arith_edge(approx_sqrt(v), a.inv, n);
  const int b = (v >= E[k]) ? k : k - 1;  // E[0] = 0 <= v: b >= 0
  return b < n ? b : -1;
}

// flat histogram slot of pair (i of A, j of B) from the FP64 coordinates;
// 0 (trash) when out of range
template <int KIND>
__device__ int slot64(const KParams &p, const PairDev &pd, int i, int j) {
  const double *A = pd.sA, *B = pd.sB;
  double ax = A[i], ay = A[(size_t)pd.nA + i], az = A[2 * (size_t)pd.nA + i];
  double bx = B[j], by = B[(size_t)pd.nB + j], bz = B[2 * (size_t)pd.nB + j];
  const double L = pd.L64;
  // L/2 halves the exponent field of L (a normal positive double)
  const int hh = pd.L32 > 0.0f ? __double2hiint(pd.L64) - (1 << 20) : -1;
  if (KIND == KMONO || KIND == KTHETA) {
    double dx = wrap64(__dsub_rn(bx, ax), L, hh), dy = wrap64(__dsub_rn(by, ay), L, hh),
           dz = wrap64(__dsub_rn(bz, az), L, hh);
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    int b = axis_bin64(p.ax[0], p.E0, p.n0, d2);
    return b < 0 ? 0 : b + 1;
  } else if (KIND == KSIGPI) {
    double dx = wrap64(__dsub_rn(bx, ax), L, hh), dy = wrap64(__dsub_rn(by, ay), L, hh),
           dz = wrap64(__dsub_rn(bz, az), L, hh);
    double s2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    double p2 = __dmul_rn(dz, dz);
    int bs = axis_bin64(p.ax[0], p.E0, p.n0, s2);
    if (bs < 0) return 0;
    int bp = axis_bin64(p.ax[1], p.E1, p.n1, p2);
    if (bp < 0) return 0;
    return (bs + 1) * p.slots1 + bp + 1;
  } else {  // KRMU, midpoint line of sight, open
    double sx = __dsub_rn(bx, ax), sy = __dsub_rn(by, ay), sz = __dsub_rn(bz, az);
    double lx = __dadd_rn(ax, bx), ly = __dadd_rn(ay, by), lz = __dadd_rn(az, bz);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(sx, sx), __dmul_rn(sy, sy)), __dmul_rn(sz, sz));
    int br = axis_bin64(p.ax[0], p.E0, p.n0, r2);
    if (br < 0) return 0;
    int bm = 0;
    if (r2 != 0.0) {
      double l2 = __dadd_rn(__dadd_rn(__dmul_rn(lx, lx), __dmul_rn(ly, ly)), __dmul_rn(lz, lz));
      double sl = __dadd_rn(__dadd_rn(__dmul_rn(sx, lx), __dmul_rn(sy, ly)), __dmul_rn(sz, lz));
      double q = __dmul_rn(sl, sl);
      double den = __dmul_rn(r2, l2);
      if (p.ax[1].mode != kArith) {
        bm = mubin64(p.E1, p.n1, q, den);
      } else if (__double2hiint(den) == 0 && __double2loint(den) == 0) {
        bm = p.n1 - 1;  // q = den = 0: every edge test holds
      } else {
        // uniform mu edges from 0: the edge nearest the FP32 estimate of
        // mu = sqrt(q / den) decides with one canonical test
        const float mu = sqrtf(approx_f32(q) / approx_f32(den));
        const int k = arith_edge(mu, p.ax[1].inv, p.n1);
        bm = (q >= __dmul_rn(p.E1[k], den)) ? k : k - 1;
        bm = min(max(bm, 0), p.n1 - 1);
      }
    }
    return (br + 1) * p.slots1 + bm + 1;
  }
}

// ---- double-float first stage of the re-test (df_stage.h): the slot of
// pair (i, j) when the stage decides it; false when it leaves a decision
// open (or an axis uses tables), the FP64 formula then decides.
template <int KIND>
__device__ bool slot_df(const KParams &p, const PairDev &pd, int i, int j, int &slot) {
  if (p.ax[0].mode != kArith || ((KIND == KSIGPI || KIND == KRMU) && p.ax[1].mode != kArith))
    return false;
  const PairDF &f = *pd.df;
  const float4 a = pd.posA[i], b = pd.posB[j], la = f.loA[i], lb = f.loB[j];
  const float pa[3] = {a.x, a.y, a.z}, pb[3] = {b.x, b.y, b.z};
  const float lav[3] = {la.x, la.y, la.z}, lbv[3] = {lb.x, lb.y, lb.z};
  const float *E0 = (const float *)p.E0df, *E1 = (const float *)p.E1df;
  int s;
  if (KIND == KMONO || KIND == KTHETA)
    s = dfs::mono_slot(pa, lav, pb, lbv, f.eta, f.Lh, f.Ll, p.ax[0].inv, E0, p.n0);
  else if (KIND == KSIGPI)
    s = dfs::sigpi_slot(pa, lav, pb, lbv, f.eta, f.Lh, f.Ll, p.ax[0].inv, E0, p.n0, p.ax[1].inv,
                        E1, p.n1);
  else
    s = dfs::rmu_slot(pa, lav, pb, lbv, f.eta, f.eta_l, f.fo2h, f.fo2l, p.ax[0].inv, E0, p.n0,
                      p.ax[1].inv, E1, p.n1);
  if (s == -2) return false;
  slot = s;
  return true;
}

}  // namespace cute

// df_stage.h -- double-float first stage of the edge re-test (host and
// device).
//
// A pair whose FP32 value lies inside an edge's error band must be binned
// as the canonical FP64 formulas of Sec. 2.2 and 3.4 bin it (the definition
// the counts are checked against).  FP64 runs at a small fraction of the
// FP32 rate on this GPU, so the re-test first forms the decision values in
// double-float (pairs of FP32 numbers, about 2^-46 relative): each object's
// frame offset x - fo is held as its FP32 value plus an FP32 remainder, the
// separation and line-of-sight components are assembled with error-free
// transformations (Knuth's TwoSum, the FMA form of Dekker's product), and
// an explicit error bound travels with each decision value.  A comparison
// whose value clears the edge by more than its bound is the canonical
// comparison; the rest (pairs within about 1e-9 of an edge, in practice the
// ones placed on edges on purpose) go to the FP64 formula.
//
// The functions here are plain arithmetic on FP32 values, compiled for the
// device (IEEE round-to-nearest intrinsics, no contraction) and for the host
// (built with -ffp-contract=off), so that the host can check them against
// FP64 on adversarial inputs.
#pragma once

#include <cmath>
#include <cstdint>

#ifdef __CUDACC__
#define CUTE_HD __host__ __device__ __forceinline__
#else
#define CUTE_HD inline
#endif

namespace cute {
namespace dfs {

// ---- IEEE FP32 operations, rounded to nearest, never contracted
CUTE_HD float add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  volatile float r = a + b;
  return r;
#endif
}
CUTE_HD float sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  volatile float r = a - b;
  return r;
#endif
}
CUTE_HD float mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  volatile float r = a * b;
  return r;
#endif
}
CUTE_HD float fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
CUTE_HD float div(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdiv_rn(a, b);
#else
  volatile float r = a / b;
  return r;
#endif
}
CUTE_HD float sqrt(float a) {
#ifdef __CUDA_ARCH__
  return __fsqrt_rn(a);
#else
  return std::sqrt(a);
#endif
}
// 1/sqrt(x), within a few ulp (the bounds below carry a 25 % margin)
CUTE_HD float rsqrt(float x) {
#ifdef __CUDA_ARCH__
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
#else
  return 1.0f / std::sqrt(x);
#endif
}
// nearest integer; NaN gives 0, out-of-range values saturate
CUTE_HD int rint_sat(float x) {
#ifdef __CUDA_ARCH__
  return __float2int_rn(x);
#else
  if (x != x) return 0;
  if (x >= 2147483520.0f) return 2147483647;
  if (x <= -2147483648.0f) return (-2147483647 - 1);
  return (int)std::nearbyint(x);
#endif
}
CUTE_HD float fmax_(float a, float b) { return a > b ? a : (b == b ? b : a); }

// ---- error-free transformations and double-float helpers
// s + e = a + b exactly (Knuth's TwoSum)
CUTE_HD void two_sum(float a, float b, float &s, float &e) {
  s = add(a, b);
  const float bp = sub(s, a);
  e = add(sub(a, sub(s, bp)), sub(b, bp));
}
// normalise (h, l): |l| <= ulp(h) / 2 afterwards, h + l unchanged
CUTE_HD void norm(float &h, float &l) {
  float a, b;
  two_sum(h, l, a, b);
  h = a;
  l = b;
}
// (h, l) += (s + e)^2, h + l left unnormalised
CUTE_HD void add_sq(float s, float e, float &h, float &l) {
  const float p = mul(s, s);
  const float pe = fma(s, s, -p);  // s^2 = p + pe exactly
  float t, te;
  two_sum(h, p, t, te);
  l = add(l, add(te, fma(add(mul(2.0f, s), e), e, pe)));
  h = t;
}
// (h, l) += (s + e)(u + w), h + l left unnormalised
CUTE_HD void add_prod(float s, float e, float u, float w, float &h, float &l) {
  const float p = mul(s, u);
  const float pe = fma(s, u, -p);
  float t, te;
  two_sum(h, p, t, te);
  l = add(l, add(te, fma(e, w, fma(s, w, fma(e, u, pe)))));
  h = t;
}
// (h, l) = (ah + al)(bh + bl) for normalised operands (al bl, below 2^-48
// of the product, left out), normalised
CUTE_HD void mul2(float ah, float al, float bh, float bl, float &h, float &l) {
  h = mul(ah, bh);
  l = fma(ah, bl, fma(al, bh, fma(ah, bh, -h)));
  norm(h, l);
}
// separation component x_j - x_i from frame offsets pos + lo, minimum image
// when Lh > 0 (the |d| > L/2 test in FP32: it differs from the FP64 one only
// for separations near L/2, beyond every reach), normalised
CUTE_HD void sep(float pb, float lb, float pa, float la, float Lh, float Ll, float &s, float &e) {
  float es;
  two_sum(pb, -pa, s, es);
  e = add(es, sub(lb, la));
  if (Lh > 0.0f && std::fabs(s) > mul(0.5f, Lh)) {
    const float sg = s > 0.0f ? -1.0f : 1.0f;
    float s2, e2;
    two_sum(s, sg * Lh, s2, e2);
    e = add(add(e, e2), sg * Ll);
    s = s2;
  }
  norm(s, e);  // lb - la is relative to the offsets, not to s
}
// line-of-sight component x_i + x_j = 2 fo + offsets, normalised
CUTE_HD void los(float pa, float la, float pb, float lb, float fo2h, float fo2l, float &u,
                 float &w) {
  float u1, w1, w2;
  two_sum(pa, pb, u1, w1);
  two_sum(u1, fo2h, u, w2);
  w = add(add(add(add(w1, w2), la), lb), fo2l);
  norm(u, w);
}
// (h + l) >= (Eh + El) given |error| <= B: 1 yes, 0 no, -1 open
CUTE_HD int ge(float h, float l, float Eh, float El, float B) {
  const float d = add(sub(h, Eh), sub(l, El));
  return d > B ? 1 : (d < -B ? 0 : -1);
}
// error bound of a sum of up to 3 squared components (each within eta) at
// value V, the larger of the sum and the edge: 2 sqrt(3 V) eta for the
// components' errors, 10 eta^2 for the second-order terms, 2^-36 V for the
// rounded sums of low parts, the 2^-48 split of the edge and the FP64
// rounding of the canonical value; 25 % margin
CUTE_HD float bound_sq(float V, float eta) {
  const float sv = mul(V, rsqrt(fmax_(V, 1e-30f)));
  return 1.25f * (3.47f * sv * eta + 10.0f * eta * eta + 1.5e-11f * V);
}
// nearest edge index of x on uniform edges from 0 (x * inv rounded), [0, n]
CUTE_HD int nearest_edge(float x, float inv, int n) {
  const int k = rint_sat(mul(x, inv));
  return k < 0 ? 0 : (k > n ? n : k);
}

// bin of a double-float squared separation (h, l) on uniform edges from 0
// (E: squared edges as hi, lo pairs; inv: 1 / bin width): -2 open, -1
// outside, else the bin.  The nearest edge k has the canonical bin at k - 1
// or k while the value is known far better than half a bin: bounds above
// 1e-4 of it stay open.
CUTE_HD int axis_bin(float inv, const float *E, int n, float h, float l, float eta) {
  const int k = nearest_edge(mul(h, rsqrt(fmax_(h, 1e-30f))), inv, n);
  const float Eh = E[2 * k], El = E[2 * k + 1];
  const float V = fmax_(h, Eh);
  const float B = bound_sq(V, eta);
  if (!(B <= 1e-4f * V)) return -2;
  if (k == 0) return 0;  // below half the first edge: bin 0 (E[0] = 0)
  const int g = ge(h, l, Eh, El, B);
  if (g < 0) return -2;
  const int b = g ? k : k - 1;
  return b < n ? b : -1;
}

// Monopole (or chord) slot: 0 outside, bin + 1 inside, -2 open.
CUTE_HD int mono_slot(const float *pa, const float *la, const float *pb, const float *lb,
                      float eta, float Lh, float Ll, float inv, const float *E0, int n0) {
  float h = 0.0f, l = 0.0f;
  for (int k = 0; k < 3; k++) {
    float s, e;
    sep(pb[k], lb[k], pa[k], la[k], Lh, Ll, s, e);
    add_sq(s, e, h, l);
  }
  norm(h, l);
  const int b = axis_bin(inv, E0, n0, h, l, eta);
  return b == -2 ? -2 : (b < 0 ? 0 : b + 1);
}

// (sigma, pi) slot with the line of sight along z (slots1 = n1 + 2).
CUTE_HD int sigpi_slot(const float *pa, const float *la, const float *pb, const float *lb,
                       float eta, float Lh, float Ll, float inv0, const float *E0, int n0,
                       float inv1, const float *E1, int n1) {
  float h = 0.0f, l = 0.0f, ph = 0.0f, pl = 0.0f;
  for (int k = 0; k < 3; k++) {
    float s, e;
    sep(pb[k], lb[k], pa[k], la[k], Lh, Ll, s, e);
    if (k < 2) add_sq(s, e, h, l);
    else add_sq(s, e, ph, pl);
  }
  norm(h, l);
  norm(ph, pl);
  const int bs = axis_bin(inv0, E0, n0, h, l, eta);
  const int bp = axis_bin(inv1, E1, n1, ph, pl, eta);
  if (bs == -2 || bp == -2) return -2;
  return (bs < 0 || bp < 0) ? 0 : (bs + 1) * (n1 + 2) + bp + 1;
}

// (r, mu) slot, mu about the midpoint line of sight (open boundary; eta_l
// bounds the line-of-sight components, fo2 = twice the frame centre).
CUTE_HD int rmu_slot(const float *pa, const float *la, const float *pb, const float *lb,
                     float eta, float eta_l, const float *fo2h, const float *fo2l, float inv0,
                     const float *E0, int n0, float inv1, const float *E1, int n1) {
  float sv[3], ev[3], u[3], w[3];
  float rh = 0.0f, rl = 0.0f;
  for (int k = 0; k < 3; k++) {
    sep(pb[k], lb[k], pa[k], la[k], 0.0f, 0.0f, sv[k], ev[k]);
    add_sq(sv[k], ev[k], rh, rl);
  }
  norm(rh, rl);
  const int br = axis_bin(inv0, E0, n0, rh, rl, eta);
  if (br == -2) return -2;
  if (br < 0) return 0;
  float l2h = 0.0f, l2l = 0.0f, slh = 0.0f, sll = 0.0f;
  for (int k = 0; k < 3; k++) {
    los(pa[k], la[k], pb[k], lb[k], fo2h[k], fo2l[k], u[k], w[k]);
    add_sq(u[k], w[k], l2h, l2l);
    add_prod(sv[k], ev[k], u[k], w[k], slh, sll);
  }
  norm(l2h, l2l);
  norm(slh, sll);
  float qh, ql, dh, dl;
  mul2(slh, sll, slh, sll, qh, ql);  // q = (s.l)^2
  mul2(rh, rl, l2h, l2l, dh, dl);    // den = r^2 l^2
  if (!(dh > 0.0f)) return -2;
  // propagated bounds: |d sl| <= sqrt3 (|s| eta_l + |l| eta) + 3 eta eta_l,
  // |d r2| and |d l2| as sums of squares, |d den| <= r2 |d l2| + l2 |d r2|
  // + |d r2||d l2|; mu = sl / sqrt(den) is then known to 1.5e-4 (far below
  // half a bin), or the decision stays open
  const float r = mul(rh, rsqrt(fmax_(rh, 1e-30f))), lm = mul(l2h, rsqrt(fmax_(l2h, 1e-30f)));
  const float dsl = 1.75f * (r * eta_l + lm * eta) + 3.0f * eta * eta_l;
  const float dr2 = 3.47f * r * eta + 10.0f * eta * eta;
  const float dl2 = 3.47f * lm * eta_l + 10.0f * eta_l * eta_l;
  const float dden = rh * dl2 + l2h * dr2 + dr2 * dl2;
  if (!(dsl <= 1e-4f * r * lm) || !(dden <= 1e-4f * dh)) return -2;
  // nearest mu edge: 0 and 1 decide nothing (every q >= 0 = m_0^2 den; the
  // top bin is closed above), an inner edge by q >= m_k^2 den
  const int k = nearest_edge(dfs::sqrt(div(qh, dh)), inv1, n1);
  int bm;
  if (k == 0) {
    bm = 0;
  } else if (k >= n1) {
    bm = n1 - 1;
  } else {
    float mh, ml;
    mul2(E1[2 * k], E1[2 * k + 1], dh, dl, mh, ml);
    const float B = 1.25f * (2.0f * std::fabs(slh) * dsl + dsl * dsl + E1[2 * k] * dden +
                             1.5e-11f * (qh + mh));
    const int g = ge(qh, ql, mh, ml, B);
    if (g < 0) return -2;
    bm = g ? k : k - 1;
  }
  return (br + 1) * (n1 + 2) + bm + 1;
}

// ---- bounds of the double-float components (host: per pair set)
// Separation component: pos + lo holds x - fo within (2^-53 + 2^-48)|x - fo|
// (the FP64 offset, then the FP32 rounding of its remainder); the FP32
// difference of the remainders and the sum with the TwoSum error add at
// most 2^-47 of the offsets and 2^-48 of the separation; the box splits as
// hi + lo within 2^-48 L.  2^-45 (xm + L) covers all of it.
inline double eta_sep(double xm, double L) { return std::ldexp(xm + L, -45) * 1.01 + 1e-37; }
// Line-of-sight component 2 fo + offsets: the remainders and the split of
// 2 fo as above, and four rounded FP32 sums of low parts (each below 2^-23
// of the offsets, the centre or the component); 2^-44 of twice the frame,
// centre and observer-frame extents covers it.
inline double eta_los(double xm, double fo_max, double abs_max) {
  return std::ldexp(2.0 * xm + 2.0 * fo_max + 2.0 * abs_max, -44) * 1.01 + 1e-37;
}

}  // namespace dfs
}  // namespace cute

// Host check of the counting kernel's FP32 binning.  Uniform edges: the
// kernel's arithmetic (count_impl.cuh: mono_arith2, sigpi_arith2,
// rmu_values2 + rmu_arith2, one element of each packed pair); other edges:
// the table path (the FP32 values of the table loop, then count_kernel.cuh's
// lut_get, axis_resolve and mu_resolve on the planner's own table and band
// arrays).  Both are replayed here in the same operation order with IEEE
// FP32 operations, the hardware reciprocal square root replaced by 1/sqrt
// perturbed by up to its documented 2^-22.9 relative error (at both
// extremes and at random), and the near-edge thresholds taken from the host
// planner (plan_build).  On
// pairs placed on and around every edge, open and periodic, every pair the
// kernel would NOT flag as near must land in the slot of the canonical FP64
// formulas (Sec. 2.2: squared separations against squared edges, minimum
// image; Sec. 3.4: mu about the midpoint line of sight).
// Prints "scenario cases flagged violations"; exits 1 on any violation.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -I include -I <csrc>
//        -I <cuda>/include fp32_band_check.cpp <csrc>/plan.cpp -L<cuda>/lib64 -lcudart
#include "cute_internal.h"

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

using namespace cute;

static const float kVFloor = 1e-30f, kMagic = 12582912.0f;
static const uint32_t kMagicBits = 0x4B400000u;
static const double kU32 = 5.9604644775390625e-08;

// ---- IEEE FP32, rounded to nearest, never contracted
static float fadd(float a, float b) { volatile float r = a + b; return r; }
static float fmul(float a, float b) { volatile float r = a * b; return r; }
static float ffma(float a, float b, float c) { return std::fma(a, b, c); }
static uint32_t bits(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }

// the hardware rsqrt: any value within 2^-22.9 of 1/sqrt(x)
static std::mt19937_64 g_rng(1210);
static int g_mode = 0;  // 0 random, 1 low extreme, 2 high extreme
// margin factor (first argument, default 1): thresholds f times as far from
// 1/2 as the planner's (f < 1 probes how much of the margin is needed)
static double g_f = 1.0;
static void shrink(AxisPlan &a) {
  a.near_at = (float)(0.5 - g_f * (0.5 - (double)a.near_at));
  a.near_c = (float)(0.5 - g_f * (0.5 - (double)a.near_c));
  a.thr_a = (float)(g_f * a.thr_a);
}
static float rsqrt_dev(float x) {
  const double r = 1.0 / std::sqrt((double)x), e = std::ldexp(1.0, -23) * 1.0717;  // 2^-22.9
  double f;
  if (g_mode == 1) f = 1.0 - e;
  else if (g_mode == 2) f = 1.0 + e;
  else f = 1.0 + e * (2.0 * std::uniform_real_distribution<double>(0, 1)(g_rng) - 1.0);
  return (float)(r * f);
}

// the hardware log2 (lg2.approx): any value within 2^-22 + 2^-23 |log2 x|
// of log2(x) -- half the bound the planner assumes; tests/test_gpu_approx.py
// finds the hardware within 0.49 of the planner's bound over every FP32
// input in [2^-60, 2^70) (as the reciprocal square root is replayed at its
// documented bound, not at the planner's)
static float lg2_dev(float x) {
  const double r = std::log2((double)x),
               e = std::ldexp(1.0, -22) + std::ldexp(1.0, -23) * std::fabs(r);
  double f;
  if (g_mode == 1) f = -e;
  else if (g_mode == 2) f = e;
  else f = e * (2.0 * std::uniform_real_distribution<double>(0, 1)(g_rng) - 1.0);
  return (float)(r + f);
}

struct Slot { int slot; float score; };

// ---- table binning
static float f32_toward(double v, bool up) {
  float f = (float)v;
  if (up && (double)f < v) f = std::nextafter(f, INFINITY);
  if (!up && (double)f > v) f = std::nextafter(f, -INFINITY);
  return f;
}
// bands of table axis `axis` f times as wide about their edges E (squared
// edges; the mu axis scales the per-class bound instead)
static void shrink_table(Plan &P, int axis, const std::vector<double> &E) {
  if (g_f == 1.0) return;
  AxisPlan &a = P.ax[axis];
  if (P.kind == KRMU && axis == 1) {
    P.mu_eps_base = (float)(g_f * P.mu_eps_base);
    return;
  }
  for (int k = 0; k < (int)E.size(); k++) {
    float &lo = P.band[2 * (a.band_off + 1 + k)], &hi = P.band[2 * (a.band_off + 1 + k) + 1];
    if (!std::isfinite(lo) || !std::isfinite(hi)) continue;
    lo = f32_toward(E[k] - g_f * (E[k] - (double)lo), false);
    hi = f32_toward(E[k] + g_f * ((double)hi - E[k]), true);
  }
}
static bool g_lut_oob = false;  // a table index outside the axis's cells
static uint32_t lut_get(const Plan &P, const AxisPlan &a, float &v) {
  v = std::fmin(v, a.vmax);  // fminf: NaN becomes vmax
  uint32_t idx;
  if (a.mode == kLutLinear) {
    idx = bits(ffma(v, a.scale, 8388608.0f)) - 0x4B000000u;
  } else {
    const int i = (int)(bits(v) >> a.shift) - a.base;
    idx = (uint32_t)std::max(i, 0);
  }
  if (idx >= (uint32_t)a.ncell) { g_lut_oob = true; return 0; }
  return P.lut[a.lut_off + idx];
}
static uint32_t axis_resolve(const Plan &P, const AxisPlan &a, float v, uint32_t e,
                             uint32_t stride, bool &near) {
  const uint32_t b = e >> kBandShift, off = e & kOffMask;
  float lo = INFINITY, hi = INFINITY;
  if (b != 0u) { lo = P.band[2 * (a.band_off + b)]; hi = P.band[2 * (a.band_off + b) + 1]; }
  const bool above = v > hi;
  near = (v >= lo) && !above;
  return above ? off + stride : off;
}
static uint32_t mu_resolve(const Plan &P, const AxisPlan &a, float mu, uint32_t e,
                           uint32_t stride, float eps, bool &near) {
  const uint32_t b = e >> kBandShift, off = e & kOffMask;
  const float m = b != 0u ? P.band[2 * (a.band_off + b)] : INFINITY;
  const float d = fadd(mu, -m);
  near = std::fabs(d) <= eps;
  return d > eps ? off + stride : off;
}
// slot and near flag of one pair from its FP32 table values (a, b)
static int table_slot(const Plan &P, float a, float b, bool &near) {
  const uint32_t stride0 = (uint32_t)P.slots1 * P.R * 4u, stride1 = (uint32_t)P.R * 4u;
  uint32_t o;
  if (P.kind == KMONO || P.kind == KTHETA) {
    const uint32_t e0 = lut_get(P, P.ax[0], a);
    o = axis_resolve(P, P.ax[0], a, e0, stride0, near);
  } else {
    const uint32_t e0 = lut_get(P, P.ax[0], a), e1 = lut_get(P, P.ax[1], b);
    bool n0, n1;
    o = axis_resolve(P, P.ax[0], a, e0, stride0, n0);
    if (P.kind == KSIGPI) {
      o += axis_resolve(P, P.ax[1], b, e1, stride1, n1);
    } else {
      uint32_t eb = bits(P.mu_eps_base) + (((e0 >> kClassShift) & 0xFu) << 23);
      float eps;
      std::memcpy(&eps, &eb, 4);
      o += mu_resolve(P, P.ax[1], b, e1, stride1, eps, n1);
    }
    near = n0 || n1;
  }
  return (int)(o / ((uint32_t)P.R * 4u));
}
static Slot mono_table(const Plan &P, const float *q, const float *n) {
  const float dx = fadd(q[0], n[0]), dy = fadd(q[1], n[1]), dz = fadd(q[2], n[2]);
  const float v = ffma(dz, dz, ffma(dy, dy, fmul(dx, dx)));
  bool near;
  const int s = table_slot(P, v, v, near);
  return {s, near ? 1.0f : 0.0f};
}
static Slot sigpi_table(const Plan &P, const float *q, const float *n) {
  const float dx = fadd(q[0], n[0]), dy = fadd(q[1], n[1]), dz = fadd(q[2], n[2]);
  bool near;
  const int s = table_slot(P, ffma(dy, dy, fmul(dx, dx)), fmul(dz, dz), near);
  return {s, near ? 1.0f : 0.0f};
}
// (r, mu) inputs of one pair: q = |x|^2 - q0 of both objects (FP64, rounded
// once to FP32, as the grid build stores them) and C_i = k (2 q_i + 4 q0)
// (FP64, rounded once, as the kernel forms it per home object)
struct RmuIn {
  float qi, qj, ci, k;
};
static RmuIn rmu_inputs(const double *xi, const double *xj, double q0, float k) {
  auto q = [&](const double *x) { return (float)(((x[0] * x[0] + x[1] * x[1]) + x[2] * x[2]) - q0); };
  RmuIn r;
  r.qi = q(xi);
  r.qj = q(xj);
  r.k = k;
  r.ci = (float)((double)k * (2.0 * (double)r.qi + 4.0 * q0));
  return r;
}
// s.l = q_j - q_i and k l.l = 2k q_j + (C_i - k r^2)
static void rmu_sl_l2(const RmuIn &in, float r2, float &sl, float &l2) {
  sl = fadd(in.qj, -in.qi);
  l2 = ffma(in.qj, 2.0f * in.k, ffma(r2, -in.k, in.ci));
}
static Slot rmu_table(const Plan &P, const float *q, const float *n, const RmuIn &in) {
  const float dx = fadd(q[0], n[0]), dy = fadd(q[1], n[1]), dz = fadd(q[2], n[2]);
  const float r2 = ffma(dz, dz, ffma(dy, dy, ffma(dx, dx, kVFloor)));
  float sl, l2;
  rmu_sl_l2(in, r2, sl, l2);
  const float mu = fmul(std::fabs(sl), rsqrt_dev(fmul(r2, l2)));
  bool near;
  const int s = table_slot(P, r2, mu, near);
  return {s, near ? 1.0f : 0.0f};
}

// one pair, monopole / chord: q neighbour offsets, n = -(home - shift)
static Slot mono_fp32(const AxisPlan &a, const float *q, const float *n) {
  const float dx = fadd(q[0], n[0]), dy = fadd(q[1], n[1]), dz = fadd(q[2], n[2]);
  const float v = ffma(dz, dz, ffma(dy, dy, ffma(dx, dx, kVFloor)));
  const float x = fmul(v, rsqrt_dev(v));
  float t = ffma(x, a.inv, a.cst);
  t = std::fmin(t, a.thi);
  const float tm = fadd(t, kMagic), fl = fadd(tm, -kMagic);
  const float h = ffma(fl, -1.0f, t);
  return {(int)(bits(tm) - kMagicBits) + 1, std::fabs(h)};
}

// log-spaced edges: t = A log2(max(v, vlo)) + (D v + B) v + C
static Slot mono_log_fp32(const AxisPlan &a, const float *q, const float *n) {
  const float dx = fadd(q[0], n[0]), dy = fadd(q[1], n[1]), dz = fadd(q[2], n[2]);
  const float v = std::fmax(ffma(dz, dz, ffma(dy, dy, fmul(dx, dx))), a.vlo);
  const float lg = lg2_dev(v), rr = rsqrt_dev(v);
  const float pv = ffma(v, ffma(v, a.ld, a.lb), a.cst);
  float t = ffma(lg, a.inv, pv);
  if (a.mode == kArithLog) t = std::fmin(t, a.thi);  // kArithLogU: no upper clamp
  const float tm = fadd(t, kMagic), fl = fadd(tm, -kMagic);
  const float h = ffma(fl, -1.0f, t);
  return {(int)(bits(tm) - kMagicBits) + 1, ffma(rr, a.thr_a, std::fabs(h))};
}

static Slot sigpi_fp32(const AxisPlan &a0, const AxisPlan &a1, int slots1, const float *q,
                       const float *n) {
  const float dx = fadd(q[0], n[0]), dy = fadd(q[1], n[1]), dz = fadd(q[2], n[2]);
  const float v0 = ffma(dy, dy, ffma(dx, dx, kVFloor));
  const float x0 = fmul(v0, rsqrt_dev(v0));
  const float t0 = std::fmin(ffma(x0, a0.inv, a0.cst), a0.thi);
  const float t1 = std::fmin(ffma(std::fabs(dz), a1.inv, a1.cst), a1.thi);
  const float tm0 = fadd(t0, kMagic), tm1 = fadd(t1, kMagic);
  const float f0 = fadd(tm0, -kMagic);
  const float h0 = ffma(f0, -1.0f, t0), h1 = ffma(fadd(tm1, -kMagic), -1.0f, t1);
  const float tc = ffma(f0, (float)slots1, tm1);
  const float g1 = fmul(h1, a1.near_scale);
  return {(int)(bits(tc) - kMagicBits) + slots1 + 1, std::fmax(std::fabs(h0), std::fabs(g1))};
}

// (r, mu) with uniform edges: axis 1 takes t = |s.l| rsqrt(r^2 k l.l) + cst
static Slot rmu_fp32(const AxisPlan &a0, const AxisPlan &a1, int slots1, const float *q,
                     const float *n, const RmuIn &in) {
  const float dx = fadd(q[0], n[0]), dy = fadd(q[1], n[1]), dz = fadd(q[2], n[2]);
  const float r2 = ffma(dz, dz, ffma(dy, dy, ffma(dx, dx, kVFloor)));
  float sl, l2;
  rmu_sl_l2(in, r2, sl, l2);
  const float rr = rsqrt_dev(r2);
  const float pl = fmul(r2, l2);
  const float t0 = std::fmin(ffma(fmul(r2, rr), a0.inv, a0.cst), a0.thi);
  const float t1 = std::fmin(ffma(std::fabs(sl), rsqrt_dev(pl), a1.cst), a1.thi);
  const float tm0 = fadd(t0, kMagic), tm1 = fadd(t1, kMagic);
  const float f0 = fadd(tm0, -kMagic);
  const float h0 = ffma(f0, -1.0f, t0), h1 = ffma(fadd(tm1, -kMagic), -1.0f, t1);
  const float tc = ffma(f0, (float)slots1, tm1);
  const float sc = std::fmax(std::fabs(h0), ffma(rr, a1.thr_a, std::fabs(h1)));
  return {(int)(bits(tc) - kMagicBits) + slots1 + 1, sc};
}

// ---- canonical FP64 (the oracle's definitions)
static double wrap(double d, double L) {
  if (L > 0) {
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
  }
  return d;
}
static int bin64(const std::vector<double> &E, double v) {
  const int n = (int)E.size() - 1;
  if (!(v >= E[0]) || !(v < E[n])) return -1;
  int b = 0;
  while (b + 1 <= n && v >= E[b + 1]) b++;
  return b;
}

struct Tally {
  long cases = 0, flagged = 0, bad = 0;
  void add(bool near, int fp32, int canon) {
    cases++;
    if (near) { flagged++; return; }
    if (fp32 != canon) {
      if (bad < 5) std::printf("  violation: fp32 slot %d canonical %d\n", fp32, canon);
      bad++;
    }
  }
};

// the library's per-component error bound (error_params): FP32 frame
// offsets within xm of the centre, periodic image shifts; for (r, mu) the
// geometry's q0 and qd from the smallest and largest |x| (grid_build)
static double rmu_q0(double rmin, double robs) { return 0.5 * (rmin * rmin + robs * robs); }
static ErrorParams eparams(double xm, double L, double rmax, double absmax, double rmin,
                           double robs = 0) {
  ErrorParams ep{0, 0, 0, 0, 0};
  ep.xm = xm;
  ep.q0 = rmu_q0(rmin, robs);
  ep.qd = 0.5 * (robs * robs - rmin * rmin) * (1.0 + 1e-12) + 1e-15 * robs * robs;
  if (L > 0) {
    const double dL = std::fabs((double)(float)L - L);
    ep.eta0 = kU32 * (3.0 * xm + 2.0 * rmax) * 1.01 + dL * 1.01 + 1e-12 * (xm + L);
  } else {
    ep.eta0 = kU32 * 2.0 * xm * 1.01 + 1e-12 * xm;
  }
  (void)absmax;
  ep.lmin = 2.0 * rmin - rmax;
  return ep;
}

static void unit(std::mt19937_64 &g, double *u) {
  std::normal_distribution<double> N(0, 1);
  double s = 0;
  for (int k = 0; k < 3; k++) { u[k] = N(g); s += u[k] * u[k]; }
  s = std::sqrt(s);
  for (int k = 0; k < 3; k++) u[k] /= s;
}

// relative offsets from an edge, both sides, across the FP32 error band
static const double kOff[] = {0.0,   1e-8, -1e-8, 1e-7, -1e-7, 4e-7, -4e-7, 1e-6,  -1e-6,
                              3e-6, -3e-6, 1e-5, -1e-5, 3e-5, -3e-5, 1e-4, -1e-4, 1e-3, -1e-3};

// FP32 offsets of a pair as the kernel sees them: q = b - fo, n = -(a - fo - S)
static void kernel_inputs(const double *a, const double *b, const double *fo, double L, float *q,
                          float *n) {
  for (int c = 0; c < 3; c++) {
    const float pa = (float)(a[c] - fo[c]), pb = (float)(b[c] - fo[c]);
    float S = 0.0f;
    if (L > 0) {
      const double d = b[c] - a[c];
      if (d > 0.5 * L) S = -(float)L;        // neighbour's image at b - L
      else if (d < -0.5 * L) S = (float)L;   // at b + L
    }
    q[c] = pb;
    n[c] = -fadd(pa, -S);
  }
}

static std::vector<double> uniform(double step, int n) {
  std::vector<double> e(n + 1);
  for (int k = 0; k <= n; k++) e[k] = k * step;
  return e;
}
static std::vector<double> logspace(double lo, double hi, int n) {
  std::vector<double> e(n + 1);
  for (int k = 0; k <= n; k++) e[k] = lo * std::pow(hi / lo, (double)k / n);
  return e;
}
static std::vector<double> squares(const std::vector<double> &e) {
  std::vector<double> E(e.size());
  for (size_t k = 0; k < e.size(); k++) E[k] = e[k] * e[k];
  return E;
}
static bool plan_ok(const std::string &m, const Plan &P, bool arith) {
  const bool got = P.ax[0].mode == kArith;
  if (m.empty() && got == arith) return true;
  std::printf("  plan: %s (arithmetic binning %d, wanted %d)\n", m.c_str(), got, arith);
  return false;
}
// binning path of a monopole / chord scenario: uniform edges by arithmetic,
// log-spaced edges by arithmetic on log2, or the tables
constexpr int kWantTable = -1;
static bool mode_ok(const std::string &m, const Plan &P, int want) {
  const int got = P.ax[0].mode;
  const bool ok = want == kWantTable ? (got == kLutLinear || got == kLutLog) : got == want;
  if (m.empty() && ok) return true;
  std::printf("  plan: %s (mode %d, wanted %d)\n", m.c_str(), got, want);
  return false;
}

// edges e (uniform from 0: the arithmetic path; otherwise the table path)
static Tally run_mono(const std::vector<double> &e, double L, double xm_spread, bool chord,
                      int want, std::mt19937_64 &g) {
  const bool arith = want != kWantTable, logm = want == kArithLog || want == kArithLogU;
  const int n = (int)e.size() - 1;
  const std::vector<double> E = squares(e);
  const double fo[3] = {chord ? 0.0 : (L > 0 ? 0.5 * L : 1234.5),
                        chord ? 0.0 : (L > 0 ? 0.5 * L : -300.25),
                        chord ? 0.97 : (L > 0 ? 0.5 * L : 77.0)};
  // unclamped log chords: points on a cap within 18 degrees of +z (pairs up to
  // 10 degrees apart stay within 0.6 of the frame centre on every axis)
  const bool cap = chord && want == kArithLogU;
  const double xm = cap ? 0.6 : (chord ? 1.0 : (L > 0 ? 0.5 * L : xm_spread + e[n]));
  Plan P;
  // (the chord counts' kernel keeps 4 KB of histogram copies per warp)
  const std::string m = plan_build(chord ? KTHETA : KMONO, e.data(), n, nullptr, 1,
                                   eparams(xm, L, e[n], 0, 0), 8192, chord ? 4096 : 12288, arith,
                                   P);
  if (!mode_ok(m, P, want)) return Tally{0, 0, 1};
  if (want == kArithLogU) {
    // every value the kernel can form, padded pairs included (up to 12
    // far^2), must take a slot inside the planner's histogram
    Tally range;
    const double vlo = P.ax[0].vlo, vmax = 12.0 * (double)P.far * (double)P.far;
    const float far_q[3] = {-P.far, -P.far, -P.far}, far_n[3] = {-P.far, -P.far, -P.far};
    for (int i = 0; i <= 200000; i++) {
      const double v = i < 200000 ? vlo * std::pow(vmax / vlo, i / 200000.0) : vmax;
      // a separation of length sqrt(v) along one axis, or the padded pair
      float q[3] = {(float)std::sqrt(v), 0.0f, 0.0f}, nn[3] = {0.0f, 0.0f, 0.0f};
      const Slot r = i < 200000 ? mono_log_fp32(P.ax[0], q, nn) : mono_log_fp32(P.ax[0], far_q, far_n);
      range.cases++;
      if (r.slot < 0 || r.slot >= P.nslots) {
        if (range.bad < 5) std::printf("  slot %d outside [0, %d) at v %g\n", r.slot, P.nslots, v);
        range.bad++;
      }
    }
    if (range.bad) return range;
  }
  if (arith) shrink(P.ax[0]);
  else shrink_table(P, 0, E);
  std::uniform_real_distribution<double> U(-1, 1);
  Tally t;
  for (int k = e[0] > 0 ? 0 : 1; k <= n; k++)
    for (double off : kOff)
      for (int rep = 0; rep < 24; rep++) {
        double a[3], b[3], u[3];
        const double s = e[k] * (1.0 + off);
        if (chord) {
          double v[3], w[3];
          unit(g, v);
          while (cap && v[2] < std::cos(18.0 * 3.141592653589793 / 180.0)) unit(g, v);
          unit(g, w);
          const double dot = w[0] * v[0] + w[1] * v[1] + w[2] * v[2];
          double wn = 0;
          for (int c = 0; c < 3; c++) { w[c] -= dot * v[c]; wn += w[c] * w[c]; }
          wn = std::sqrt(wn);
          const double ang = 2 * std::asin(std::min(1.0, s / 2));
          for (int c = 0; c < 3; c++) {
            a[c] = v[c];
            b[c] = std::cos(ang) * v[c] + std::sin(ang) * w[c] / wn;
          }
        } else {
          unit(g, u);
          for (int c = 0; c < 3; c++) {
            a[c] = L > 0 ? std::fmod(fo[c] + 0.5 * L * U(g) + 10 * L, L) : fo[c] + xm_spread * U(g);
            b[c] = a[c] + u[c] * s;
            if (L > 0) { b[c] = std::fmod(b[c] + 10 * L, L); if (b[c] >= L) b[c] = 0; }
          }
        }
        float q[3], nn[3];
        kernel_inputs(a, b, fo, L, q, nn);
        double dd[3];
        for (int c = 0; c < 3; c++) dd[c] = wrap(b[c] - a[c], L);
        const int cb = bin64(E, (dd[0] * dd[0] + dd[1] * dd[1]) + dd[2] * dd[2]);
        const int canon = cb < 0 ? -1 : cb + 1;
        const Slot r = logm ? mono_log_fp32(P.ax[0], q, nn)
                            : (arith ? mono_fp32(P.ax[0], q, nn) : mono_table(P, q, nn));
        const int fp32 = (r.slot >= 1 && r.slot <= n) ? r.slot : -1;
        t.add(logm ? r.score >= P.ax[0].near_c
                   : (arith ? r.score >= P.ax[0].near_at : r.score > 0.0f),
              fp32, canon);
      }
  return t;
}

static Tally run_sigpi(const std::vector<double> &e0, const std::vector<double> &e1, double L,
                       bool arith, std::mt19937_64 &g) {
  const int n0 = (int)e0.size() - 1, n1 = (int)e1.size() - 1;
  const std::vector<double> E0 = squares(e0), E1 = squares(e1);
  const double fo[3] = {0.5 * L, 0.5 * L, 0.5 * L};
  Plan P;
  const std::string m = plan_build(KSIGPI, e0.data(), n0, e1.data(), n1,
                                   eparams(0.5 * L, L, std::max(e0[n0], e1[n1]), 0, 0), 8192, 12288,
                                   true, P);
  if (!plan_ok(m, P, arith)) return Tally{0, 0, 1};
  if (arith) {
    shrink(P.ax[0]);
    shrink(P.ax[1]);
    P.ax[1].near_scale = (float)((double)P.ax[0].near_at / (double)P.ax[1].near_at);
  } else {
    shrink_table(P, 0, E0);
    shrink_table(P, 1, E1);
  }
  std::uniform_real_distribution<double> U(-1, 1), U01(0, 1);
  Tally t;
  for (int axis = 0; axis < 2; axis++)
    for (int k = (axis ? e1 : e0)[0] > 0 ? 0 : 1; k <= (axis ? n1 : n0); k++)
      for (double off : kOff)
        for (int rep = 0; rep < 16; rep++) {
          const double ed = (axis ? e1[k] : e0[k]) * (1.0 + off);
          const double sig = axis ? U01(g) * e0[n0] : ed, pi = axis ? ed : U01(g) * e1[n1];
          const double phi = 6.283185307179586 * U01(g);
          const double o3[3] = {sig * std::cos(phi), sig * std::sin(phi), U(g) > 0 ? pi : -pi};
          double a[3], b[3];
          for (int c = 0; c < 3; c++) {
            a[c] = std::fmod(fo[c] + 0.5 * L * U(g) + 10 * L, L);
            b[c] = std::fmod(a[c] + o3[c] + 10 * L, L);
            if (b[c] >= L) b[c] = 0;
          }
          float q[3], nn[3];
          kernel_inputs(a, b, fo, L, q, nn);
          double dd[3];
          for (int c = 0; c < 3; c++) dd[c] = wrap(b[c] - a[c], L);
          const int bs = bin64(E0, dd[0] * dd[0] + dd[1] * dd[1]), bp = bin64(E1, dd[2] * dd[2]);
          const int canon = (bs < 0 || bp < 0) ? -1 : (bs + 1) * (n1 + 2) + bp + 1;
          const Slot r = arith ? sigpi_fp32(P.ax[0], P.ax[1], P.slots1, q, nn) : sigpi_table(P, q, nn);
          const int s0i = r.slot / P.slots1, s1i = r.slot % P.slots1;
          const int fp32 = (s0i >= 1 && s0i <= n0 && s1i >= 1 && s1i <= n1) ? r.slot : -1;
          t.add(arith ? r.score >= P.ax[0].near_at : r.score > 0.0f, fp32, canon);
        }
  return t;
}

// (r, mu) on a light-cone-like region: objects around centre fo (observer
// at the origin), extent xm about fo
static Tally run_rmu(const double *fo, double xm, double rmin, double robs, double absmax,
                     const std::vector<double> &e0, int n1, std::vector<double> rs, bool arith,
                     std::mt19937_64 &g) {
  const int n0 = (int)e0.size() - 1;
  std::vector<double> e1(n1 + 1);
  for (int k = 0; k <= n1; k++) e1[k] = (double)k / n1;
  const std::vector<double> E0 = squares(e0), M = squares(e1);
  Plan P;
  const ErrorParams ep = eparams(xm, 0, e0[n0], absmax, rmin, robs);
  const std::string m = plan_build(KRMU, e0.data(), n0, e1.data(), n1, ep, 8192, 12288, true, P);
  if (!plan_ok(m, P, arith) || (arith && P.ax[1].mode != kArith)) return Tally{0, 0, 1};
  if (arith) {
    shrink(P.ax[0]);
    shrink(P.ax[1]);
  } else {
    shrink_table(P, 0, E0);
    shrink_table(P, 1, M);
  }
  const float thr = std::fmin(P.ax[0].near_at, P.ax[1].near_c);
  std::uniform_real_distribution<double> U(-1, 1);
  Tally t;
  for (double r : rs)
    for (int k = 0; k <= n1; k++)
      for (double off : kOff)
        for (int rep = 0; rep < 3; rep++) {
          // x_i in the shell, far enough inside it that x_j = x_i + s is too
          double xi[3], tt[3], ri = 0;
          do {
            for (int c = 0; c < 3; c++) xi[c] = fo[c] + (xm - 210.0) * U(g);
            ri = std::sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
          } while (ri < rmin + 201.0 || ri > robs - 201.0);
          unit(g, tt);
          const double mm = std::min(std::max(e1[k] * (1.0 + off), 0.0), 1.0);
          const double rr = (rep == 0 && k == 0) ? r * (1.0 + off) : r;
          double s[3] = {0, 0, 0};
          for (int it = 0; it < 8; it++) {
            double l[3], ln = 0;
            for (int c = 0; c < 3; c++) { l[c] = 2 * xi[c] + s[c]; ln += l[c] * l[c]; }
            ln = std::sqrt(ln);
            double dot = 0;
            for (int c = 0; c < 3; c++) dot += tt[c] * l[c] / ln;
            double tp[3], tn = 0;
            for (int c = 0; c < 3; c++) { tp[c] = tt[c] - dot * l[c] / ln; tn += tp[c] * tp[c]; }
            tn = std::sqrt(tn);
            for (int c = 0; c < 3; c++)
              s[c] = rr * (mm * l[c] / ln + std::sqrt(std::max(0.0, 1 - mm * mm)) * tp[c] / tn);
          }
          double xj[3];
          for (int c = 0; c < 3; c++) xj[c] = xi[c] + s[c];
          // canonical
          const double sx = xj[0] - xi[0], sy = xj[1] - xi[1], sz = xj[2] - xi[2];
          const double lx = xi[0] + xj[0], ly = xi[1] + xj[1], lz = xi[2] + xj[2];
          const double r2 = (sx * sx + sy * sy) + sz * sz;
          int canon = -1;
          const int br = bin64(E0, r2);
          if (br >= 0) {
            int bm = 0;
            if (r2 != 0.0) {
              const double l2 = (lx * lx + ly * ly) + lz * lz;
              const double sl = (sx * lx + sy * ly) + sz * lz;
              const double qv = sl * sl, den = r2 * l2;
              for (int mi = 1; mi <= n1 - 1; mi++)
                if (qv >= M[mi] * den) bm = mi;
            }
            canon = (br + 1) * (n1 + 2) + bm + 1;
          }
          // the kernel's inputs
          float q[3], nn[3];
          kernel_inputs(xi, xj, fo, 0.0, q, nn);
          const RmuIn in = rmu_inputs(xi, xj, ep.q0, P.ax[1].lsc);
          const Slot res = arith ? rmu_fp32(P.ax[0], P.ax[1], P.slots1, q, nn, in)
                                 : rmu_table(P, q, nn, in);
          const int s0i = res.slot / P.slots1, s1i = res.slot % P.slots1;
          const int fp32 = (s0i >= 1 && s0i <= n0 && s1i >= 1 && s1i <= n1) ? res.slot : -1;
          t.add(arith ? res.score >= thr : res.score > 0.0f, fp32, canon);
        }
  return t;
}

// ---- integer lattices: integer coordinates and edges make the canonical
// FP64 values exact, so many pairs sit exactly on an edge; each such pair
// must be flagged (or land in its slot all the same).  Every pair of the
// points is checked; `ties` counts the exact ties.
static std::vector<double> lattice_pts(std::mt19937_64 &g, int n, const double lo[3],
                                       const double hi[3]) {
  std::vector<double> p(3 * n);
  for (int i = 0; i < n; i++)
    for (int c = 0; c < 3; c++) p[3 * i + c] = std::uniform_int_distribution<int>((int)lo[c], (int)hi[c] - 1)(g);
  return p;
}

// logm: monopole edges 1, 2, 4, ..., 32 (log-spaced: arithmetic on log2)
static Tally run_lattice_mono_sigpi(bool sigpi, bool arith, bool periodic, std::mt19937_64 &g,
                                    long &ties, bool logm = false) {
  const std::vector<double> e0 =
      sigpi ? (arith ? uniform(1.0, 9) : std::vector<double>{0, 1, 2, 3, 4, 6, 9})
            : (logm ? std::vector<double>{1, 2, 4, 8, 16}
                    : (arith ? uniform(1.0, 13) : std::vector<double>{0, 1, 2, 3, 5, 8, 13}));
  const std::vector<double> e1 = arith ? uniform(1.0, 7) : std::vector<double>{0, 1, 3, 5, 7};
  const int n0 = (int)e0.size() - 1, n1 = sigpi ? (int)e1.size() - 1 : 1;
  const std::vector<double> E0 = squares(e0), E1 = squares(e1);
  const double L = periodic ? 40.0 : 0.0;
  const double fo[3] = {periodic ? 20.0 : 1000.37, periodic ? 20.0 : -299.81, periodic ? 20.0 : 77.5};
  const double lo[3] = {periodic ? 0.0 : 985.0, periodic ? 0.0 : -315.0, periodic ? 0.0 : 62.0};
  const double hi[3] = {periodic ? 40.0 : 1016.0, periodic ? 40.0 : -284.0, periodic ? 40.0 : 93.0};
  const double xm = periodic ? 20.0 : 16.0;
  Plan P;
  const std::string m = sigpi ? plan_build(KSIGPI, e0.data(), n0, e1.data(), n1,
                                           eparams(xm, L, std::max(e0[n0], e1[n1]), 0, 0), 8192,
                                           12288, true, P)
                              : plan_build(KMONO, e0.data(), n0, nullptr, 1,
                                           eparams(xm, L, e0[n0], 0, 0), 8192, 12288, true, P);
  if (logm ? !mode_ok(m, P, kArithLog) : !plan_ok(m, P, arith)) return Tally{0, 0, 1};
  if (arith || logm) {
    shrink(P.ax[0]);
    if (sigpi) {
      shrink(P.ax[1]);
      P.ax[1].near_scale = (float)((double)P.ax[0].near_at / (double)P.ax[1].near_at);
    }
  } else {
    shrink_table(P, 0, E0);
    if (sigpi) shrink_table(P, 1, E1);
  }
  // (exact ties at 1, 4, 16, 64, 256 are rarer than at every integer: more points)
  const std::vector<double> x = lattice_pts(g, logm ? 900 : 320, lo, hi);
  const int n = (int)x.size() / 3;
  Tally t;
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++) {
      float q[3], nn[3];
      kernel_inputs(&x[3 * i], &x[3 * j], fo, L, q, nn);
      double dd[3];
      for (int c = 0; c < 3; c++) dd[c] = wrap(x[3 * j + c] - x[3 * i + c], L);
      int canon;
      Slot r;
      if (!sigpi) {
        const double d2 = (dd[0] * dd[0] + dd[1] * dd[1]) + dd[2] * dd[2];
        for (int k = 1; k <= n0; k++) ties += d2 == E0[k];
        const int cb = bin64(E0, d2);
        canon = cb < 0 ? -1 : cb + 1;
        r = logm ? mono_log_fp32(P.ax[0], q, nn)
                 : (arith ? mono_fp32(P.ax[0], q, nn) : mono_table(P, q, nn));
        const int fp32 = (r.slot >= 1 && r.slot <= n0) ? r.slot : -1;
        t.add(logm ? r.score >= P.ax[0].near_c
                   : (arith ? r.score >= P.ax[0].near_at : r.score > 0.0f),
              fp32, canon);
      } else {
        const double sg2 = dd[0] * dd[0] + dd[1] * dd[1], pi2 = dd[2] * dd[2];
        for (int k = 1; k <= n0; k++) ties += sg2 == E0[k];
        for (int k = 1; k <= n1; k++) ties += pi2 == E1[k];
        const int bs = bin64(E0, sg2), bp = bin64(E1, pi2);
        canon = (bs < 0 || bp < 0) ? -1 : (bs + 1) * (n1 + 2) + bp + 1;
        r = arith ? sigpi_fp32(P.ax[0], P.ax[1], P.slots1, q, nn) : sigpi_table(P, q, nn);
        const int s0i = r.slot / P.slots1, s1i = r.slot % P.slots1;
        const int fp32 = (s0i >= 1 && s0i <= n0 && s1i >= 1 && s1i <= n1) ? r.slot : -1;
        t.add(arith ? r.score >= P.ax[0].near_at : r.score > 0.0f, fp32, canon);
      }
    }
  return t;
}

// (r, mu) far from the observer, with pairs at exactly mu = 1/2:
// s = 2 m s0, l = x_i + x_j = 2 q (1, 1, 0), s0 at 60 degrees to (1, 1, 0)
static Tally run_lattice_rmu(bool arith, std::mt19937_64 &g, long &ties) {
  const std::vector<double> e0 = arith ? uniform(1.0, 13) : std::vector<double>{0, 1, 2, 3, 5, 8, 13};
  const int n0 = (int)e0.size() - 1, n1 = 4;
  std::vector<double> e1(n1 + 1);
  for (int k = 0; k <= n1; k++) e1[k] = (double)k / n1;
  const std::vector<double> E0 = squares(e0), M = squares(e1);
  std::vector<double> x;
  const int s0[4][3] = {{1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}};
  for (int q = 300; q < 340; q += 8)
    for (int m = 1; m <= 4; m++)
      for (auto &v : s0)
        for (int sg = -1; sg <= 1; sg += 2)
          for (int c = 0; c < 3; c++) x.push_back((c < 2 ? q : 0) + sg * m * v[c]);
  const double lo[3] = {300, 300, -10}, hi[3] = {341, 341, 11};
  const std::vector<double> rp = lattice_pts(g, 200, lo, hi);
  x.insert(x.end(), rp.begin(), rp.end());
  const double fo[3] = {320.25, 319.5, 0.125};
  double xm = 0, absmax = 0, rmin = 1e300, robs = 0;
  for (size_t i = 0; i < x.size(); i += 3) {
    double a2 = 0;
    for (int c = 0; c < 3; c++) {
      xm = std::max(xm, std::fabs(x[i + c] - fo[c]));
      absmax = std::max(absmax, std::fabs(x[i + c]));
      a2 += x[i + c] * x[i + c];
    }
    rmin = std::min(rmin, std::sqrt(a2));
    robs = std::max(robs, std::sqrt(a2));
  }
  Plan P;
  const ErrorParams ep = eparams(xm, 0, e0[n0], absmax, rmin, robs);
  const std::string m = plan_build(KRMU, e0.data(), n0, e1.data(), n1, ep, 8192, 12288, true, P);
  if (!plan_ok(m, P, arith) || (arith && P.ax[1].mode != kArith)) return Tally{0, 0, 1};
  if (arith) {
    shrink(P.ax[0]);
    shrink(P.ax[1]);
  } else {
    shrink_table(P, 0, E0);
    shrink_table(P, 1, M);
  }
  const float thr = std::fmin(P.ax[0].near_at, P.ax[1].near_c);
  const int n = (int)x.size() / 3;
  Tally t;
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++) {
      const double *xi = &x[3 * i], *xj = &x[3 * j];
      const double sx = xj[0] - xi[0], sy = xj[1] - xi[1], sz = xj[2] - xi[2];
      const double lx = xi[0] + xj[0], ly = xi[1] + xj[1], lz = xi[2] + xj[2];
      const double r2 = (sx * sx + sy * sy) + sz * sz;
      for (int k = 1; k <= n0; k++) ties += r2 == E0[k];
      int canon = -1;
      const int br = bin64(E0, r2);
      if (br >= 0) {
        int bm = 0;
        if (r2 != 0.0) {
          const double l2 = (lx * lx + ly * ly) + lz * lz;
          const double sl = (sx * lx + sy * ly) + sz * lz;
          const double qv = sl * sl, den = r2 * l2;
          for (int mi = 1; mi <= n1 - 1; mi++) {
            if (qv >= M[mi] * den) bm = mi;
            ties += qv == M[mi] * den;
          }
        }
        canon = (br + 1) * (n1 + 2) + bm + 1;
      }
      float q[3], nn[3];
      kernel_inputs(xi, xj, fo, 0.0, q, nn);
      const RmuIn in = rmu_inputs(xi, xj, ep.q0, P.ax[1].lsc);
      const Slot res = arith ? rmu_fp32(P.ax[0], P.ax[1], P.slots1, q, nn, in)
                             : rmu_table(P, q, nn, in);
      const int s0i = res.slot / P.slots1, s1i = res.slot % P.slots1;
      const int fp32 = (s0i >= 1 && s0i <= n0 && s1i >= 1 && s1i <= n1) ? res.slot : -1;
      t.add(arith ? res.score >= thr : res.score > 0.0f, fp32, canon);
    }
  return t;
}

int main(int argc, char **argv) {
  if (argc > 1) g_f = std::atof(argv[1]);
  std::mt19937_64 g(20121008);
  long bad = 0;
  auto report = [&](const char *name, const Tally &t) {
    std::printf("%s %ld %ld %ld\n", name, t.cases, t.flagged, t.bad);
    bad += t.bad;
  };
  const std::vector<double> rs_u = {0.4, 2.0, 4.999, 5.0, 12.5, 33.0, 77.0, 120.0, 180.0, 199.9, 200.0};
  const std::vector<double> r_log = logspace(1.0, 200.0, 20);
  std::vector<double> rs_l = rs_u;
  rs_l.insert(rs_l.end(), r_log.begin(), r_log.end());
  // chords of 64 log-spaced angles 0.01 .. 10 degrees (the w(theta) workload)
  std::vector<double> chords = logspace(0.01, 10.0, 64);
  for (double &c : chords) c = 2.0 * std::sin(0.5 * c * 3.141592653589793 / 180.0);
  const double fo[3] = {1250.0, 1083.0, 625.0};
  for (g_mode = 0; g_mode < 3; g_mode++) {
    char nm[64];
    std::snprintf(nm, sizeof nm, "mono_periodic_r%d", g_mode);
    report(nm, run_mono(uniform(5.0, 30), 2000.0, 0, false, kArith, g));
    std::snprintf(nm, sizeof nm, "mono_periodic_small_r%d", g_mode);
    report(nm, run_mono(uniform(5.0, 40), 1000.0, 0, false, kArith, g));
    std::snprintf(nm, sizeof nm, "mono_open_r%d", g_mode);
    report(nm, run_mono(uniform(2.5, 40), 0.0, 1400.0, false, kArith, g));
    std::snprintf(nm, sizeof nm, "chord_r%d", g_mode);
    report(nm, run_mono(uniform(0.0027, 64), 0.0, 0, true, kArith, g));
    std::snprintf(nm, sizeof nm, "sigpi_periodic_r%d", g_mode);
    report(nm, run_sigpi(uniform(3.0, 50), uniform(3.0, 50), 1500.0, true, g));
    std::snprintf(nm, sizeof nm, "rmu_lightcone_r%d", g_mode);
    report(nm, run_rmu(fo, 1250.0, 1000.0, 2500.0, 2500.0, uniform(5.0, 40), 40, rs_u, true, g));
    // the table path (edges not uniform from 0)
    std::snprintf(nm, sizeof nm, "table_mono_periodic_r%d", g_mode);
    report(nm, run_mono(logspace(0.1, 150.0, 20), 2000.0, 0, false, kWantTable, g));
    std::snprintf(nm, sizeof nm, "table_mono_open_r%d", g_mode);
    report(nm, run_mono(logspace(1.0, 200.0, 16), 0.0, 1400.0, false, kWantTable, g));
    std::snprintf(nm, sizeof nm, "table_chord_r%d", g_mode);
    report(nm, run_mono(chords, 0.0, 0, true, kWantTable, g));
    // log-spaced edges by arithmetic on log2 of the square
    std::snprintf(nm, sizeof nm, "log_mono_periodic_r%d", g_mode);
    report(nm, run_mono(logspace(0.1, 150.0, 20), 2000.0, 0, false, kArithLog, g));
    std::snprintf(nm, sizeof nm, "log_mono_open_r%d", g_mode);
    report(nm, run_mono(logspace(1.0, 200.0, 16), 0.0, 1400.0, false, kArithLog, g));
    std::snprintf(nm, sizeof nm, "log_chord_r%d", g_mode);
    report(nm, run_mono(chords, 0.0, 0, true, kArithLogU, g));
    std::snprintf(nm, sizeof nm, "table_sigpi_periodic_r%d", g_mode);
    report(nm, run_sigpi(logspace(0.5, 60.0, 15), uniform(2.0, 30), 1500.0, false, g));
    std::snprintf(nm, sizeof nm, "table_rmu_lightcone_r%d", g_mode);
    report(nm, run_rmu(fo, 1250.0, 1000.0, 2500.0, 2500.0, r_log, 10, rs_l, false, g));
  }
  // integer lattices ("name cases flagged violations", then "name_ties count")
  for (g_mode = 0; g_mode < 3; g_mode++) {
    struct L { const char *name; int kind; bool arith, periodic; };
    const L ls[] = {{"lattice_mono_arith_periodic", 0, true, true},
                    {"lattice_mono_arith_open", 0, true, false},
                    {"lattice_mono_table_periodic", 0, false, true},
                    {"lattice_mono_table_open", 0, false, false},
                    {"lattice_sigpi_arith_periodic", 1, true, true},
                    {"lattice_sigpi_table_periodic", 1, false, true},
                    {"lattice_rmu_arith", 2, true, false},
                    {"lattice_rmu_table", 2, false, false},
                    {"lattice_mono_log_periodic", 3, false, true},
                    {"lattice_mono_log_open", 3, false, false}};
    for (const L &l : ls) {
      long ties = 0;
      char nm[80];
      std::snprintf(nm, sizeof nm, "%s_r%d", l.name, g_mode);
      report(nm, l.kind == 2 ? run_lattice_rmu(l.arith, g, ties)
                             : run_lattice_mono_sigpi(l.kind == 1, l.arith, l.periodic, g, ties,
                                                      l.kind == 3));
      std::printf("%s_ties %ld\n", nm, ties);
    }
  }
  if (g_lut_oob) {
    std::printf("table index outside the table\n");
    bad++;
  }
  return bad ? 1 : 0;
}

// plan.cpp -- host planning for the counting kernels: per-axis lookup tables
// with proven FP32 error bands, arithmetic binning of uniform edges, and the
// home chunks and neighbour stencil of a pair set.
//
// Binning (the bin of each pair's separation, Sec. 3.1).  For non-uniform
// edges the kernels compute each separation in FP32 and look its squared value up
// in a table.  A table cell is CLEAN when every FP32 value it holds, widened
// by the error bound err(v) of the FP32 computation, lies strictly between
// the same two bin edges, so the FP32 result bins the pair exactly as the
// FP64 canonical formula does.  Other cells are DIRTY and name the single
// edge whose band meets them; pairs that land within that band are re-tested
// in FP64.  Both the table geometry (linear or logarithmic in v) and its size
// are chosen here by the expected fraction of pairs landing in dirty cells.
//
// Neighbour search (Sec. 3.3): catalog A is cut, row of cells by row, into
// home chunks; each chunk is paired with the rows of neighbour cells of the
// stencil around it.  Within a row the neighbour cells are contiguous in the
// cell-sorted order, so each (chunk, neighbour row) is at most a few
// contiguous ranges of catalog B (work.cu turns them into work items).
#include "cute_internal.h"

#include <thread>

#include <algorithm>
#include <cmath>
#include <cstring>

namespace cute {

static const double kU = 5.9604644775390625e-08;  // 2^-24, FP32 unit roundoff

static float f32_down(double x) {
  float f = (float)x;
  if ((double)f > x) f = std::nextafter(f, -INFINITY);
  return f;
}
static float f32_up(double x) {
  float f = (float)x;
  if ((double)f < x) f = std::nextafter(f, INFINITY);
  return f;
}
static uint32_t fbits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}
static float bitsf(uint32_t u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

Plan::~Plan() {
  if (d_lut) cudaFree(d_lut);
  if (d_band) cudaFree(d_band);
  if (d_E0) cudaFree(d_E0);
  if (d_E1) cudaFree(d_E1);
  if (d_E0df) cudaFree(d_E0df);
  if (d_E1df) cudaFree(d_E1df);
}

// ------------------------------------------------------------------ error models
// Error of an FP32 sum of c squared components whose components carry an
// absolute error of at most eta0 + u|delta|, relative to the FP64 canonical
// value of the same quantity.  Derivation: |d32^2 - d^2| <= eta(2|d| + eta)
// per component, sum |d_k| <= sqrt(c v); the c FP32 roundings of the sum of
// squares add at most (c+1) u v; the FP64 canonical value differs from the
// exact one by less than 4e-16 v.  The result is doubled as a safety margin.
struct SqErr {
  int c;
  double eta0;
  double operator()(double v) const {
    v = std::max(v, 0.0);
    double sv = std::sqrt(v);
    double eta = eta0 + kU * sv * 1.0001;
    double e = eta * (2.0 * std::sqrt((double)c) * sv + c * eta) + (c + 1) * kU * v * 1.01 +
               4e-16 * v;
    return 2.0 * e + 1e-300;
  }
};

// A generic error model: err(v) for v-type axes, constant for mu.
struct AxisErr {
  bool constant = false;
  double cst = 0;
  SqErr sq{3, 0};
  double operator()(double v) const { return constant ? cst : sq(v); }
};

// ------------------------------------------------------------------ one axis table
struct AxisSpec {
  std::vector<double> E;     // edges in the looked-up quantity (squared, or mu)
  std::vector<int> decision; // indices k of E that are decision boundaries
  int nb = 0;                // bins
  AxisErr err;
  double density_p = 0;      // density model v^p for choosing the table
  double vtop = 0;           // largest value that can be in range
  bool mu = false;           // mu axis: no out-of-range slot
};

struct AxisTable {
  AxisPlan p;
  std::vector<uint32_t> cells;       // entries (offset units filled in later)
  std::vector<int> slot;             // slot of clean cells (-1 dirty)
  std::vector<int> edge;             // edge of dirty cells (-1 none, -2 always)
  std::vector<double> cell_hi;       // upper value of each cell
  double dirty_frac = 1.0;
};

// value interval [lo, hi] of table cell c
static void cell_range(const AxisPlan &p, int c, double &lo, double &hi) {
  if (p.mode == kLutLinear) {
    double s = (double)p.scale;
    lo = (c == 0) ? 0.0 : (c - 0.5) / s;
    hi = (c == p.ncell - 1) ? INFINITY : (c + 0.5) / s;
    lo = (c == 0) ? 0.0 : lo * (1 - 1e-12);
    hi = hi * (1 + 1e-12);
  } else {
    if (c == 0) lo = 0.0;
    else lo = bitsf((uint32_t)(c + p.base) << p.shift);
    if (c == p.ncell - 1) hi = INFINITY;
    else hi = bitsf((((uint32_t)(c + p.base + 1)) << p.shift) - 1u);
  }
}

// slot of a value known to lie in [lo, hi] with no decision edge inside
static int slot_of(const AxisSpec &a, double v) {
  if (a.mu) {
    int s = 1;
    for (int k : a.decision)
      if (a.E[k] <= v) s++;
    return s;  // 1 .. nb
  }
  int cnt = 0;
  for (size_t k = 0; k < a.E.size(); k++)
    if (a.E[k] <= v) cnt++;
  return cnt;  // 0: below the first edge, nb+1: at or above the last
}

static double dens_int(double p, double a, double b) {
  // integral of v^p over [a, b], p > -1
  a = std::max(a, 0.0);
  if (!(b > a)) return 0.0;
  return (std::pow(b, p + 1) - std::pow(a, p + 1)) / (p + 1);
}

static void classify(const AxisSpec &a, AxisTable &t) {
  const AxisPlan &p = t.p;
  t.cells.assign(p.ncell, 0);
  t.slot.assign(p.ncell, -1);
  t.edge.assign(p.ncell, -1);
  t.cell_hi.assign(p.ncell, 0);
  double tot = dens_int(a.density_p, 0.0, a.vtop), dirty = 0;
  for (int c = 0; c < p.ncell; c++) {
    double lo, hi;
    cell_range(p, c, lo, hi);
    t.cell_hi[c] = hi;
    double tlo = lo - a.err(lo);
    double thi = std::isinf(hi) ? INFINITY : hi + a.err(hi);
    int found = -1, nfound = 0;
    for (int k : a.decision) {
      if (a.E[k] >= tlo && a.E[k] <= thi) {
        found = k;
        nfound++;
      }
    }
    if (nfound == 0) {
      t.slot[c] = slot_of(a, lo);
    } else {
      t.edge[c] = (nfound == 1) ? found : -2;
      double dhi = std::isinf(hi) ? a.vtop : std::min(hi, a.vtop);
      dirty += dens_int(a.density_p, lo, dhi);
    }
  }
  t.dirty_frac = tot > 0 ? dirty / tot : 1.0;
}

static bool make_linear(const AxisSpec &a, int ncell, AxisTable &t) {
  // cover [0, vmax] with ncell cells; vmax above the top decision band
  double top = a.vtop + a.err(a.vtop);
  double vmax = top * (1.0 + 4.0 / ncell) + 1e-30;
  float vmaxf = f32_up(vmax);
  float scale = f32_down((double)(ncell - 1) / (double)vmaxf);
  // the largest index must stay inside the table: rne(vmax*scale) <= ncell-1
  while (std::nearbyint((double)vmaxf * (double)scale) > ncell - 1)
    scale = std::nextafter(scale, 0.0f);
  if (!(scale > 0) || (double)vmaxf * scale >= 4194304.0) return false;
  // the table ends at the cell that holds vmax (and every clamped value)
  ncell = (int)std::nearbyint((double)vmaxf * (double)scale) + 1;
  t.p = AxisPlan();
  t.p.mode = kLutLinear;
  t.p.ncell = ncell;
  t.p.vmax = vmaxf;
  t.p.scale = scale;
  classify(a, t);
  return true;
}

static bool make_log(const AxisSpec &a, int budget, int m, AxisTable &t) {
  // first positive decision edge
  double first = INFINITY;
  for (int k : a.decision)
    if (a.E[k] > 0) first = std::min(first, a.E[k]);
  if (!std::isfinite(first)) return false;
  double low = (first - a.err(first)) * 0.5;
  if (!(low > 1e-37)) return false;
  double top = a.vtop + a.err(a.vtop);
  float vmaxf = f32_up(top * 1.05 + 1e-30);
  int shift = 23 - m;
  int base = (int)(fbits(f32_down(low)) >> shift);
  int ncell = (int)(fbits(vmaxf) >> shift) - base + 1;
  if (ncell < 2 || ncell > budget) return false;
  t.p = AxisPlan();
  t.p.mode = kLutLog;
  t.p.ncell = ncell;
  t.p.vmax = vmaxf;
  t.p.shift = shift;
  t.p.base = base;
  classify(a, t);
  return true;
}

static AxisTable best_table(const AxisSpec &a, int budget) {
  AxisTable best, cur;
  best.dirty_frac = 2.0;
  if (make_linear(a, budget, cur) && cur.dirty_frac < best.dirty_frac) best = cur;
  for (int m = 12; m >= 3; m--) {
    if (make_log(a, budget, m, cur)) {
      if (cur.dirty_frac < best.dirty_frac) best = cur;
      break;  // the largest m that fits is the finest log table
    }
  }
  return best;
}

// Band (lo, hi) of decision edge k: a value v32 < lo is certainly below the
// edge, v32 > hi certainly above.  lo + err(lo) < E and hi - err(hi) > E.
static void edge_band(const AxisSpec &a, int k, double &lo, double &hi) {
  double E = a.E[k];
  double e = a.err(E);
  lo = E - 1.0001 * e;
  hi = E + 1.0001 * e;
  for (int it = 0; it < 64 && hi - a.err(hi) <= E; it++) hi = E + 1.01 * a.err(hi) + 1e-300;
  for (int it = 0; it < 64 && lo + a.err(E) >= E; it++) lo = E - 1.01 * (E - lo) - 1e-300;
}

// ------------------------------------------------------------------ uniform edges
// Uniform edges e_k = e_0 + k delta allow binning by arithmetic: with
// x = sqrt(v) (or |dz|, or mu) and t = (x - e_0)/delta, the bin is floor(t).
// The canonical decision for edge k compares the FP64 value with e_k^2, i.e.
// x with sqrt(fl(e_k^2)), which sits within db of t = k.  The FP32 t carries
// the error of x (from the squared value's bound err(v), the documented
// 2 ulp of rsqrtf and the product), of the FP32 constants and of the FMA.
static bool uniform_edges(const double *e, int n, double &delta) {
  delta = (e[n] - e[0]) / n;
  if (!(delta > 0)) return false;
  for (int k = 0; k <= n; k++)
    if (std::fabs(e[k] - (e[0] + k * delta)) > 1e-9 * delta) return false;
  return true;
}

// ARITH parameters of a value axis (x = sqrt(v), or x = |v| when lin).
// squared: the canonical boundaries are sqrt(fl(e_k^2)); mu: m_k itself.
static bool make_arith(const double *e, int n, const AxisErr &err, double eta0, bool squared,
                       bool is_mu, bool lin, AxisPlan &p) {
  double delta;
  if (!uniform_edges(e, n, delta)) return false;
  // the kernels clamp t only from above: with x >= 0 and e_0 = 0, t >= -1/2
  // (slot >= 1) holds without a lower clamp; other edges take the tables
  if (e[0] != 0.0) return false;
  const double inv = 1.0 / delta, c = -e[0] / delta;
  double db = 0;
  for (int k = 0; k <= n; k++) {
    long double b = squared ? sqrtl((long double)(e[k] * e[k])) : (long double)e[k];
    db = std::max(db, (double)fabsl((b - (long double)e[0]) / (long double)delta - k));
  }
  db += 1e-12 * n;
  const float inv32 = (float)inv;
  const float c32 = (float)(c - 0.5);
  // rounding of the FP32 constants, per unit of x and absolute
  const double dinv = std::fabs((double)inv32 - inv);
  const double dc = std::fabs((double)c32 - (c - 0.5));
  p = AxisPlan();
  p.mode = kArith;
  p.nb = n;
  p.inv = inv32;
  p.cst = c32;
  // non-decision edges are clamped to half-integers (never near): x >= 0
  // makes edge 0 moot when e_0 = 0, and mu never leaves [0, 1]
  const bool lo_decides = !(is_mu || e[0] == 0.0);
  p.tlo = lo_decides ? -1.0f : 0.0f;                // t - 1/2 >= -1  (t >= -1/2)
  p.thi = is_mu ? (float)(n - 1) : (float)n;        // t - 1/2 <= n (mu: n - 1)
  if (is_mu) {
    p.thr_a = 0;  // filled by the caller (depends on the r bound)
    p.thr_b = (float)(db + 4.0 * kU * n + dc + 1e-6);
    return true;
  }
  // sup over x in [0, e_n + delta] of the error of t, in t units
  double T = 0;
  const double xmax = e[n] + delta;
  for (int i = 0; i <= 4000; i++) {
    double x = xmax * std::pow(10.0, -12.0 * (1.0 - i / 4000.0));  // log grid to xmax
    if (i == 0) x = 0;
    double v = x * x;
    double dx;
    if (lin) {
      dx = 2.0 * (eta0 + kU * x * 1.0001);  // |dz|: the component bound, doubled
    } else {
      double ev = err(v);
      dx = (x > 0) ? std::min(ev / x, std::sqrt(ev)) : std::sqrt(ev);
    }
    if (!lin) dx += 6.0 * kU * x + 1e-11;  // rsqrtf (2 ulp), product, tiny-value guard
    double t = x * inv + c;
    double Tt = dx * inv + x * dinv + dc + kU * (std::fabs(t) + 1.0) + db;
    T = std::max(T, Tt);
  }
  // T is taken with the doubled error of the separation (SqErr) or of the
  // component (|dz|): that factor 2 is the margin over the analysed bound
  // (a host check replaying the kernel's arithmetic on pairs around every
  // edge finds no miss with thresholds at 0.3 of this distance, the first
  // ones near a quarter)
  p.thr_a = 0;
  p.thr_b = (float)(T + 1e-6);
  return p.thr_b < 0.2f;
}

// ------------------------------------------------------------------ log-spaced edges
// Edges uniform in a logarithm -- log r bins (ln r = ln(v)/2), and angles
// log-spaced in theta binned on squared chords c^2, where theta = 2 asin(c/2)
// makes ln theta = ln(c^2)/2 + g(c^2/4) with g(y) = ln(asin(sqrt y)/sqrt y)
// = y/6 + 11 y^2/180 + ... smooth and small -- take
//   t(v) = A log2(v) + (D v + B) v + C,  v the squared separation,
// fitted (least squares, long double) so that t(E_k) = k - 1/2 at the
// canonical boundaries E_k = fl(e_k^2); db is the largest miss there,
// measured with the FP32 constants the kernel uses.  With t monotone, a
// pair whose FP32 t lies farther than db + (its error) from every
// half-integer is binned as the canonical formula bins it.
//
// The error of the FP32 t at v (in t units) is
//   t'(v) err(v) + A e_lg + (rounding of the three FMAs) + db,
// with err(v) the squared separation's bound (SqErr, already doubled),
// e_lg(v) = 2^-21 + 2^-22 |log2 v| for the hardware log2 (lg2.approx: an
// absolute part, and about two ulp of the FP32 result; a GPU test measures
// it over every FP32 input of the range in use), and t'(v) = A/(v ln 2) +
// |B| + 2|D| v.  Its A/(v ln 2) err(v) part falls as 1/sqrt(v): the bound is taken
// as thr_a / sqrt(v) + thr_b, thr_b the parts that do not fall and thr_a the
// smallest constant that covers the rest at every v (sampled on a fine log
// grid), raised by the relative error of the FP32 v (the kernel takes
// 1/sqrt(v) from the FP32 v) and rsqrtf's 2 ulp.
// v is clamped below at vlo, where t(vlo) = -1 (slot 0, far from edge 0).
static bool solve_ld(int m, long double M[4][5], long double *x) {
  for (int c = 0; c < m; c++) {
    int piv = c;
    for (int r = c + 1; r < m; r++)
      if (fabsl(M[r][c]) > fabsl(M[piv][c])) piv = r;
    if (!(fabsl(M[piv][c]) > 0)) return false;
    for (int k = 0; k <= m; k++) std::swap(M[c][k], M[piv][k]);
    for (int r = 0; r < m; r++) {
      if (r == c) continue;
      const long double f = M[r][c] / M[c][c];
      for (int k = c; k <= m; k++) M[r][k] -= f * M[c][k];
    }
  }
  for (int c = 0; c < m; c++) x[c] = M[c][m] / M[c][c];
  return true;
}

static long double logt(const AxisPlan &p, long double v) {
  return (long double)p.inv * log2l(v) + ((long double)p.ld * v + (long double)p.lb) * v +
         (long double)p.cst;
}

static bool make_logarith(const double *e, int n, const SqErr &err, AxisPlan &p) {
  if (n < 2 || !(e[0] > 0)) return false;
  std::vector<long double> E(n + 1);
  for (int k = 0; k <= n; k++) E[k] = (long double)(e[k] * e[k]);  // canonical FP64 squares
  // unknowns: A (log2 v), C (1), B (v), D (v^2); fewer with few edges
  const int m = std::min(4, n + 1);
  long double sc[4] = {0, 0, 0, 0};
  auto col = [&](int j, long double v) -> long double {
    return j == 0 ? log2l(v) : (j == 1 ? 1.0L : (j == 2 ? v : v * v));
  };
  for (int j = 0; j < m; j++)
    for (int k = 0; k <= n; k++) sc[j] = std::max(sc[j], fabsl(col(j, E[k])));
  long double M[4][5] = {};
  for (int k = 0; k <= n; k++) {
    long double f[4];
    for (int j = 0; j < m; j++) f[j] = col(j, E[k]) / sc[j];
    for (int a = 0; a < m; a++) {
      for (int b = 0; b < m; b++) M[a][b] += f[a] * f[b];
      M[a][m] += f[a] * ((long double)k - 0.5L);
    }
  }
  long double x[4] = {0, 0, 0, 0};
  if (!solve_ld(m, M, x)) return false;
  p = AxisPlan();
  p.mode = kArithLog;
  p.nb = n;
  p.inv = (float)(x[0] / sc[0]);
  p.cst = (float)(x[1] / sc[1]);
  p.lb = m > 2 ? (float)(x[2] / sc[2]) : 0.0f;
  p.ld = m > 3 ? (float)(x[3] / sc[3]) : 0.0f;
  if (!(p.inv > 0)) return false;
  // the miss at the boundaries, with the FP32 constants
  long double db = 0;
  for (int k = 0; k <= n; k++) db = std::max(db, fabsl(logt(p, E[k]) - ((long double)k - 0.5L)));
  if (!(db < 0.01L)) return false;
  // vlo: t(vlo) = -1, below E_0 (bisection on the monotone model)
  long double lo = E[0] * 1e-12L, hi = E[0];
  if (!(logt(p, lo) < -1.0L)) return false;
  for (int it = 0; it < 200; it++) {
    const long double mid = sqrtl(lo * hi);
    if (logt(p, mid) < -1.0L) lo = mid; else hi = mid;
  }
  p.vlo = (float)hi;
  const double vlo = (double)p.vlo;
  if (!(logt(p, vlo) > -1.2L && logt(p, vlo) < -0.8L)) return false;
  p.thi = (float)n;
  // the value at which t reaches n + 1/2 (beyond it the clamp holds t at n)
  long double vtop = E[n];
  while (logt(p, vtop) < (long double)n + 0.5L && vtop < 1e30L) vtop *= 1.01L;
  const double A = p.inv, B = std::fabs((double)p.lb), D = std::fabs((double)p.ld);
  auto elg = [](double v) {
    return std::ldexp(1.0, -21) + std::ldexp(1.0, -22) * std::fabs(std::log2(v));
  };
  // FP32 rounding of the three FMAs: u of |D v + B|, u of |(.) v + C| and
  // u of |t|, the latter two below |C| + B v + D v^2 + n + 2
  auto rnd = [&](double v) {
    return kU * (std::fabs((double)p.cst) + B * v + D * v * v + n + 2.0) * 2.0 * 1.01 +
           kU * (D * v + B) * v * 1.01;
  };
  const double vt = (double)vtop;
  double thr_b = (B + 2.0 * D * vt) * err(vt) + A * elg(vt) + rnd(vt) + (double)db + 1e-7;
  // rounding parts that do not fall with v: the err(v)/v constant part
  // 2 ((c+1) u + 2 sqrt3 u + 4e-16) through A / ln 2
  thr_b += A / std::log(2.0) * 2.0 * (4.0 * kU * 1.01 + 2.0 * std::sqrt(3.0) * kU * 1.0001 + 4e-16);
  double thr_a = 0, maxrel = 0;
  for (int i = 0; i <= 4000; i++) {
    const double v = vlo * std::pow(vt / vlo, i / 4000.0);
    const double T = (A / (v * std::log(2.0)) + B + 2.0 * D * v) * err(v) + A * elg(v) + rnd(v) +
                     (double)db + 1e-7;
    thr_a = std::max(thr_a, (T - thr_b) * std::sqrt(v));
    maxrel = std::max(maxrel, err(v) / v);
  }
  thr_a = std::max(thr_a, 0.0) * (1.0 + maxrel + 4.0 * kU) * 1.0001;
  p.thr_a = (float)thr_a;
  p.thr_b = (float)thr_b;
  p.near_c = f32_down(0.5 - thr_b - std::ldexp(1.0, -22));
  // the bands must stay narrow where pairs are binned: at E_0
  return thr_a / std::sqrt((double)E[0]) + thr_b < 0.2;
}

// Chords with log-spaced edges may drop the upper clamp of t (one
// instruction per pair) when every t the kernel can form fits in spare
// histogram slots above the last bin.  The values the kernel forms lie in
// [vlo, vmax], vmax the squared separation of a padded home slot (+far on
// every axis) and a padded tile row (-far): 12 far^2, with far = 1.25 (xm +
// reach) -- every padded pair is then more than the reach apart (each axis
// at least far - xm > reach / sqrt 3) -- and the fitted t, sampled over that
// range, stays in [-1.2, tmax]; slots up to rint(tmax + 1/2) + 2 hold them
// all (the FP32 t is within a few 1e-5 of the model).  Returns the slots
// needed (0 when it does not apply).
static int logarith_top(const AxisPlan &p, double xm, double reach, float &far_out) {
  const double far = 1.25 * (xm + reach) * (1.0 + 1e-6) + 1e-30;
  const float farf = f32_up(far);
  const long double vmax = 12.0L * (long double)farf * (long double)farf * (1.0L + 1e-6L);
  long double tmax = -1e30L, tmin = 1e30L;
  const long double vlo = (long double)p.vlo;
  if (!(vmax > vlo)) return 0;
  for (int i = 0; i <= 20000; i++) {
    const long double v = vlo * powl(vmax / vlo, (long double)i / 20000.0L);
    const long double t = logt(p, v);
    tmax = std::max(tmax, t);
    tmin = std::min(tmin, t);
  }
  if (!(tmin >= -1.2L) || !(tmax < 4000.0L)) return 0;
  far_out = farf;
  return (int)floorl(tmax + 0.5L) + 4;
}

// ------------------------------------------------------------------ mu bound
// Error of the kernel's FP32 mu about the midpoint line of sight (Sec. 2.1),
// as eps(r) = a / r + b for a pair at separation r.  The kernel forms
//   s.l = q_j - q_i            (q = |x|^2 - q0, rounded once from FP64;
//                               |x_j|^2 - |x_i|^2 = (x_j - x_i).(x_j + x_i)),
//   k l^2 = k (2 q_j) + (C_i - k r^2),  C_i = k (2 q_i + 4 q0) rounded once
//                              (|l|^2 = 2|x_i|^2 + 2|x_j|^2 - r^2),
//   mu k^-1/2 = |s.l| rsqrt(r^2 k l^2),
// with r^2 from the FP32 separation.  Then
//   * s.l: |dq_i| + |dq_j| <= 2 u qd (each q rounded to nearest once), over
//     r |l| >= r lmin: 2 u qd / lmin per unit of 1/r, taken x 1.25 (the
//     bound is rigorous; the margin absorbs the first-order products), and
//     the subtraction's rounding, u |s.l| <= u r |l| (in the budget below);
//   * r^2: mu ~ (r^2)^-1/2 takes half its relative error, err(r^2) / 2r^2
//     (SqErr, already twice the first-order bound): 2 sqrt3 eta0 / r +
//     2 sqrt3 u, the square's own rounding inside the budget;
//   * k l^2: half its relative error eps_l, from the roundings of C_i (u of
//     |2 q_i + 4 q0| <= 2 qd + 4 q0), of the two q's (2 u qd each, doubled),
//     of the two FMAs (u of |C_i - k r^2| and u of k |l|^2 <= 4 k (q0 + qd))
//     and r^2's error, over k |l|^2 >= k lmin^2; taken x 1.1;
//   * 40 u for the other roundings (s.l, k, the product r^2 k l^2, rsqrtf's
//     documented 2 ulp, the final FMA and r^2's rounding: about 10 u).
// False when no lower bound of |l| exists (catalogs around the observer).
static bool mu_bound(const ErrorParams &ep, double rmax, double &a, double &b) {
  if (!(ep.lmin > 0)) return false;
  const double s3 = std::sqrt(3.0);
  const double P = 2.0 * ep.qd + 4.0 * ep.q0;
  const SqErr r2err{3, ep.eta0};
  const double eps_l = (kU * P + 4.0 * kU * ep.qd + kU * (P + rmax * rmax) +
                        4.0 * kU * (ep.q0 + ep.qd) + r2err(rmax * rmax)) /
                       (ep.lmin * ep.lmin) * (1.0 + 1e-6);
  a = 2.0 * s3 * ep.eta0 * (1.0 + 1e-5) + 1.25 * 2.0 * kU * ep.qd / ep.lmin;
  b = 2.0 * s3 * kU + 0.55 * eps_l + 40 * kU + 1e-12;
  return std::isfinite(a) && std::isfinite(b);
}

// ------------------------------------------------------------------ plan
std::string plan_build(int kind, const double *e0, int n0, const double *e1, int n1,
                       const ErrorParams &ep, int lut_budget_words, size_t hist_budget_bytes,
                       bool allow_arith, Plan &out) {
  const bool two_d = (kind == KRMU || kind == KSIGPI);
  if (n0 + 3 > 4095 || (two_d && n1 + 3 > 4095)) return "too many bins on one axis";
  out.kind = kind;
  out.n0 = n0;
  out.n1 = two_d ? n1 : 1;
  out.slots1 = two_d ? n1 + 2 : 1;
  out.nslots = (n0 + 2) * out.slots1;
  // copies of the per-warp histogram: as many (<= 32, power of 2) as fit
  int R = 32;
  while (R > 1 && (size_t)out.nslots * R * 4 > hist_budget_bytes) R >>= 1;
  if ((size_t)out.nslots * 4 > hist_budget_bytes) return "too many bins for the shared-memory histogram";
  out.R = R;

  out.E0.resize(n0 + 1);
  for (int k = 0; k <= n0; k++) out.E0[k] = e0[k] * e0[k];
  if (two_d) {
    out.E1.resize(n1 + 1);
    for (int k = 0; k <= n1; k++) out.E1[k] = e1[k] * e1[k];
  } else {
    out.E1.assign(2, 0.0);
  }
  // the squared edges as FP32 hi + lo (E - hi is exact in FP64; lo holds
  // it to 2^-24, so hi + lo is within 2^-48 E of E)
  auto split = [](const std::vector<double> &E, std::vector<float> &out2) {
    out2.resize(2 * E.size());
    for (size_t k = 0; k < E.size(); k++) {
      const float h = (float)E[k];
      out2[2 * k] = h;
      out2[2 * k + 1] = (float)(E[k] - (double)h);
    }
  };
  split(out.E0, out.E0df);
  split(out.E1, out.E1df);

  // axis specifications
  AxisSpec A0, A1;
  A0.E = out.E0;
  A0.nb = n0;
  for (int k = 0; k <= n0; k++)
    if (A0.E[k] > 0) A0.decision.push_back(k);
  A0.vtop = A0.E[n0];
  A0.err.constant = false;
  if (kind == KSIGPI) {
    A0.err.sq = SqErr{2, ep.eta0};
    A0.density_p = 0.0;  // sigma^2 of pairs spread in a plane: flat
    A1.E = out.E1;
    A1.nb = n1;
    for (int k = 0; k <= n1; k++)
      if (A1.E[k] > 0) A1.decision.push_back(k);
    A1.vtop = A1.E[n1];
    A1.err.sq = SqErr{1, ep.eta0};
    A1.density_p = -0.5;  // pi^2 of pairs spread along a line
  } else {
    A0.err.sq = SqErr{3, ep.eta0};
    A0.density_p = 0.5;   // d^2 of pairs spread in a volume
    if (kind == KTHETA) A0.density_p = 0.0;  // chord^2 of pairs on a sphere
  }

  // uniform edges on every axis: arithmetic binning, no tables
  if (allow_arith) {
    AxisPlan P0, P1;
    bool ok = false;
    if (kind == KMONO || kind == KTHETA) {
      ok = make_arith(e0, n0, A0.err, ep.eta0, true, false, false, P0);
    } else if (kind == KSIGPI) {
      ok = make_arith(e0, n0, A0.err, ep.eta0, true, false, false, P0) &&
           make_arith(e1, n1, A1.err, ep.eta0, true, false, true, P1);
    } else if (kind == KRMU) {
      ok = make_arith(e0, n0, A0.err, ep.eta0, true, false, false, P0) &&
           make_arith(e1, n1, A0.err, ep.eta0, false, true, false, P1);
      if (ok) {
        // mu bound in t units: n_mu * eps(r), eps(r) = a / r + b (mu_bound
        // below), without the final doubling: the squared separation's
        // bound is itself twice the first-order one, the q term is rigorous
        // (x 1.25), and the 40 u rounding budget is four times the kernel's
        double a = 0, b = 0;
        const bool fin = mu_bound(ep, e0[n0], a, b);
        double nmu = n1 / (e1[n1] - e1[0]);
        P1.thr_a = (float)(nmu * a * 1.0001);
        P1.thr_b = (float)((double)P1.thr_b + nmu * b * 1.0001);
        // the kernel forms k l^2 with k = 1/n_mu^2 in FP32 (its rounding,
        // u/2 relative in mu, is inside the rounding budget)
        P1.lsc = (float)(1.0 / (nmu * nmu));
        ok = fin && (double)P1.thr_b < 0.2;
      }
    }
    if (ok) {
      P0.near_at = f32_down(0.5 - (double)P0.thr_b);
      P1.near_at = f32_down(0.5 - (double)P1.thr_b);
      P1.near_c = f32_down(0.5 - (double)P1.thr_b - std::ldexp(1.0, -22));
      // (sigma, pi): |h1| * near_scale >= near_at of axis 0 whenever
      // |h1| >= near_at of axis 1 (one threshold for both axes)
      if (kind == KSIGPI) P1.near_scale = f32_up((double)P0.near_at / (double)P1.near_at);
      out.ax[0] = P0;
      out.ax[1] = two_d ? P1 : AxisPlan();
      out.lut.clear();
      out.band.assign(2, 0.0f);
      out.dirty_frac[0] = out.dirty_frac[1] = 0;
      return "";
    }
    // log-spaced monopole or chord edges: arithmetic on log2 of the square
    AxisPlan PL;
    if ((kind == KMONO || kind == KTHETA) && make_logarith(e0, n0, A0.err.sq, PL)) {
      // (not for weighted counts, planned with a 1 KB histogram budget: their
      // float-float column per slot and lane would grow with the spare slots)
      if (kind == KTHETA && hist_budget_bytes >= 4096) {
        float far = 0;
        const int need = logarith_top(PL, ep.xm, e0[n0], far);
        int Ru = 32;
        while (Ru > 1 && (size_t)need * Ru * 4 > hist_budget_bytes) Ru >>= 1;
        // only when as many histogram copies fit as with the clamp
        if (need > 0 && Ru >= out.R && (size_t)need * Ru * 4 <= kOffMask) {
          PL.mode = kArithLogU;
          out.nslots = need;
          out.far = far;
        }
      }
      out.ax[0] = PL;
      out.ax[1] = AxisPlan();
      out.lut.clear();
      out.band.assign(2, 0.0f);
      out.dirty_frac[0] = out.dirty_frac[1] = 0;
      return "";
    }
  }

  // mu on the tables: the bound a / r + b of mu_bound, doubled.  It grows
  // as 1/r: each r slot carries an error class c (bound = base * 2^c, base =
  // the bound at r_max), r slots below r_floor = max(first nonzero edge,
  // r_max / 40) are always re-tested in FP64, and the mu table is classified
  // with the largest bound in use.
  std::vector<int> always_slot(n0 + 2, 0), cls_slot(n0 + 2, 0);
  if (kind == KRMU) {
    double ma = 0, mb = 0;
    if (!mu_bound(ep, e0[n0], ma, mb)) return "(r, mu) catalogs too close to the observer";
    auto eps_at = [&](double r) {
      return r > 0 ? 2.0 * (ma / r + mb) + 1e-12 : INFINITY;
    };
    double r_floor = e0[n0] / 40.0;
    for (int k = 1; k <= n0; k++)
      if (e0[k] > 0) { r_floor = std::max(r_floor, e0[k]); break; }
    double minw = 1.0;
    for (int k = 0; k < n1; k++) minw = std::min(minw, e1[k + 1] - e1[k]);
    const float base = f32_up(eps_at(e0[n0]));
    out.mu_eps_base = base;
    double eps_max = base;
    for (int b = 0; b < n0; b++) {
      if (e0[b] < r_floor) { always_slot[b + 1] = 1; continue; }
      double e = eps_at(e0[b]);
      int c = 0;
      while (c < 15 && (double)base * std::ldexp(1.0, c) < e) c++;
      if ((double)base * std::ldexp(1.0, c) < e) { always_slot[b + 1] = 1; continue; }
      cls_slot[b + 1] = c;
      eps_max = std::max(eps_max, (double)base * std::ldexp(1.0, c));
    }
    if (!(eps_max < 0.25 * minw)) return "mu error bound too wide for the mu bins";
    A1.mu = true;
    A1.E.assign(e1, e1 + n1 + 1);
    A1.nb = n1;
    for (int k = 1; k < n1; k++) A1.decision.push_back(k);
    A1.vtop = 1.0;
    A1.err.constant = true;
    A1.err.cst = eps_max;
    A1.density_p = 0.0;
  }

  int budget0 = two_d ? lut_budget_words / 2 : lut_budget_words;
  AxisTable T0 = best_table(A0, budget0), T1;
  if (T0.p.ncell == 0) return "could not build the axis-0 lookup table";
  if (two_d) {
    T1 = best_table(A1, lut_budget_words - T0.p.ncell);
    if (T1.p.ncell == 0) return "could not build the axis-1 lookup table";
  }
  out.dirty_frac[0] = T0.dirty_frac;
  out.dirty_frac[1] = two_d ? T1.dirty_frac : 0.0;

  // bands: index 0 none (never near, never above), k+1 for edge k,
  // nb+2 always near; FP32, rounded outward.  mu bands hold the FP32 edge
  // twice: the kernel compares |mu - edge| with the pair's r-slot bound.
  out.band.clear();
  auto bands = [&](const AxisSpec &a, AxisPlan &p) {
    p.band_off = (int)out.band.size() / 2;
    p.nband = a.nb + 3;
    out.band.push_back(INFINITY);
    out.band.push_back(INFINITY);
    for (int k = 0; k <= a.nb; k++) {
      double lo = 0, hi = 0;
      bool dec = std::find(a.decision.begin(), a.decision.end(), k) != a.decision.end();
      if (!dec) {
        out.band.push_back(INFINITY);  // not a decision edge: never met
        out.band.push_back(INFINITY);
        continue;
      }
      if (a.mu) {
        out.band.push_back((float)a.E[k]);
        out.band.push_back((float)a.E[k]);
        continue;
      }
      edge_band(a, k, lo, hi);
      out.band.push_back(f32_down(lo));
      out.band.push_back(f32_up(hi));
    }
    out.band.push_back(-INFINITY);
    out.band.push_back(INFINITY);
  };
  bands(A0, T0.p);
  T0.p.nb = n0;
  if (two_d) {
    bands(A1, T1.p);
    T1.p.nb = n1;
    if (kind == KRMU)
      for (int c = 0; c < T1.p.ncell; c++)
        if (T1.edge[c] == -2) return "mu table too coarse for the mu bins";
  }

  // entries
  const uint32_t stride0 = (uint32_t)out.slots1 * R * 4, stride1 = (uint32_t)R * 4;
  if ((size_t)out.nslots * R * 4 > kOffMask) return "histogram too large";
  auto encode = [&](const AxisSpec &a, AxisTable &t, uint32_t stride, bool rmu_r) {
    const uint32_t always_band = (uint32_t)(a.nb + 2) << kBandShift;
    for (int c = 0; c < t.p.ncell; c++) {
      if (t.edge[c] == -2) {
        t.cells[c] = always_band;
      } else if (t.edge[c] == -1) {
        int sl = t.slot[c];
        t.cells[c] = (uint32_t)sl * stride;
        if (rmu_r && sl >= 1 && sl <= a.nb) {
          if (always_slot[sl]) t.cells[c] = always_band;
          else t.cells[c] |= (uint32_t)cls_slot[sl] << kClassShift;
        }
      } else {
        int k = t.edge[c];
        int below = k, above = k + 1;  // slots on either side of edge k
        t.cells[c] = ((uint32_t)(k + 1) << kBandShift) | ((uint32_t)below * stride);
        if (rmu_r) {
          int lo = std::min(below, a.nb + 1), hi = std::min(above, a.nb + 1);
          if (always_slot[lo] || always_slot[hi]) t.cells[c] = always_band;
          else t.cells[c] |= (uint32_t)std::max(cls_slot[lo], cls_slot[hi]) << kClassShift;
        }
      }
    }
  };
  encode(A0, T0, stride0, kind == KRMU);
  if (two_d) encode(A1, T1, stride1, false);

  out.lut.clear();
  T0.p.lut_off = 0;
  out.lut.insert(out.lut.end(), T0.cells.begin(), T0.cells.end());
  out.ax[0] = T0.p;
  if (two_d) {
    T1.p.lut_off = (int)out.lut.size();
    out.lut.insert(out.lut.end(), T1.cells.begin(), T1.cells.end());
    out.ax[1] = T1.p;
  } else {
    out.ax[1] = AxisPlan();
  }
  return "";
}

// The neighbour cull keeps a row whose FP32 gap vector g to the home box
// (computed from FP32 frame offsets) has |g|^2 <= cull_r2.  Each component
// of a pair's separation in FP32 differs from the exact one by at most
// e = u (3 xm + 2 L): the neighbour's offset (u xm), the home's offset
// (u xm), its image x - S in FP32 (u (xm + L)) and the FP32 box size
// (u L); the gap of a pair's neighbour is at most the FP32 separation, so
// |g| <= |s| + sqrt(3) e, and the gap's own FP32 arithmetic (one
// subtraction, a product and two fused adds) adds under 5u relative.
// Radii (r + 2e)(1 + 1e-5), squared and rounded up, therefore keep every
// pair with |s| <= r: the cull drops only pairs beyond the last edge.
void cull_params(const std::vector<DescInfo> &dis, const cute_pair_desc *d, int n, KParams &p) {
  double xm = 0.0, L = 0.0, r0 = 0.0, r1 = 0.0;
  for (const DescInfo &di : dis) {
    xm = std::max(xm, std::max(di.g->xmax[0], std::max(di.g->xmax[1], di.g->xmax[2])));
    if (di.g->periodic) L = std::max(L, di.g->L);
  }
  for (int i = 0; i < n; i++) {
    r0 = std::max(r0, d[i].edges0[d[i].n0]);
    if (d[i].kind == CUTE_SIGMA_PI) r1 = std::max(r1, d[i].edges1[d[i].n1]);
  }
  const double e = kU * (3.0 * xm + 2.0 * L);
  auto up = [](double v) {
    float f = (float)v;
    return (double)f < v ? std::nextafter(f, INFINITY) : f;
  };
  const double c0 = (r0 + 2.0 * e) * (1.0 + 1e-5);
  p.cull_r2 = up(c0 * c0);
  p.cull_pi = d[0].kind == CUTE_SIGMA_PI ? up((r1 + 2.0 * e) * (1.0 + 1e-5)) : INFINITY;
}

// ------------------------------------------------------------------ work decomposition
// A home chunk spans at most this many cells of its row: on a periodic
// axis the chunk's neighbour x-range (its cells widened by k on each side)
// must not wrap onto itself, and on an open axis wider runs only add
// candidates.
int chunks_maxrun(const Geometry &g) {
  const int nx = g.nc[0], kx = g.k[0];
  return g.periodic ? std::max(1, nx - 2 * kx) : kx + 1;
}

// Each row of cells is cut into chunks of exactly home_chunk objects (the
// last one of the row shorter); a chunk may straddle cells, so every lane's
// home slots stay occupied, and its neighbour x-range is taken from its
// first and last cells.
// The rows of cells [r0, r1) (row = cy + ny * cz), in row order.
static void chunks_rows(const Geometry &g, const int32_t *csA, int home_chunk, int64_t r0,
                        int64_t r1, std::vector<int4> &out) {
  const int nx = g.nc[0], ny = g.nc[1];
  const int maxrun = chunks_maxrun(g);
  auto cell = [&](int x, int y, int z) { return ((int64_t)z * ny + y) * nx + x; };
  for (int64_t r = r0; r < r1; r++) {
    {
      const int cy = (int)(r % ny), cz = (int)(r / ny);
      const int row_lo = csA[cell(0, cy, cz)], row_hi = csA[cell(nx - 1, cy, cz) + 1];
      int pos = row_lo, cxc = 0;
      while (pos < row_hi) {
        while (csA[cell(cxc, cy, cz) + 1] <= pos) cxc++;  // cell of the chunk's first object
        const int cx0 = cxc;
        int h1 = std::min(pos + home_chunk, row_hi);
        int cx1 = cx0;
        while (cx1 + 1 < nx && csA[cell(cx1, cy, cz) + 1] < h1) cx1++;  // cell of its last object
        if (cx1 - cx0 + 1 > maxrun) {  // cap the span: stop at the end of a cell
          cx1 = cx0 + maxrun - 1;
          h1 = csA[cell(cx1, cy, cz) + 1];
        }
        out.push_back(make_int4(pos, h1, cx0 | (cx1 << 16), cy | (cz << 16)));
        pos = h1;
      }
    }
  }
}

void chunks_build(const Geometry &g, const int32_t *csA, int home_chunk,
                  std::vector<int4> &out) {
  const int64_t rows = (int64_t)g.nc[1] * g.nc[2];
  const int64_t cells = rows * g.nc[0];
  // large grids: contiguous row ranges on a few threads, joined in order
  int nt = 1;
  if (cells >= (1 << 18)) {
    nt = (int)std::min<int64_t>(8, std::max<unsigned>(1u, std::thread::hardware_concurrency()));
    nt = (int)std::min<int64_t>(nt, rows);
  }
  if (nt <= 1) {
    chunks_rows(g, csA, home_chunk, 0, rows, out);
    return;
  }
  std::vector<std::vector<int4>> part(nt);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; t++)
    th.emplace_back([&, t] { chunks_rows(g, csA, home_chunk, rows * t / nt, rows * (t + 1) / nt, part[t]); });
  for (auto &x : th) x.join();
  size_t tot = 0;
  for (auto &v : part) tot += v.size();
  out.reserve(out.size() + tot);
  for (auto &v : part) out.insert(out.end(), v.begin(), v.end());
}

// Objects in cells |d| apart on an axis are at least (|d| - 1) a apart
// there, so a row can only reach kxr cells along x: the in-range region is a
// ball of radius need (shape 1) or a disk of radius need[0] in x-y times a
// slab in z (shape 2).  The half stencil of an auto count keeps the home row
// (whose earlier cells the chunk order covers) and the rows after it.
void stencil_build(const Geometry &g, bool is_auto, bool full_stencil, int shape,
                   const double need[3], std::vector<int4> &out) {
  const int kx = g.k[0], ky = g.k[1], kz = g.k[2];
  for (int dz = -kz; dz <= kz; dz++) {
    for (int dy = -ky; dy <= ky; dy++) {
      const bool self_row = (dz == 0 && dy == 0);
      int kxr = kx;
      if (shape != kShapeBox) {
        const double shrink = 1.0 - 1e-9;
        double gy = std::max(std::abs(dy) - 1, 0) * g.a[1] * shrink / need[1];
        double gz = std::max(std::abs(dz) - 1, 0) * g.a[2] * shrink / need[2];
        double rem = 1.0 - gy * gy - (shape == kShapeBall ? gz * gz : 0.0);
        if (shape == kShapeDiskSlab && gz >= 1.0) continue;
        if (rem <= 0.0) continue;
        kxr = std::min(kx, (int)std::ceil(std::sqrt(rem) * need[0] * (1.0 + 1e-9) / g.a[0]));
      }
      if (is_auto && !full_stencil && !self_row && (dz < 0 || (dz == 0 && dy < 0))) continue;
      out.push_back(make_int4(dy, dz, kxr, self_row ? 1 : 0));
    }
  }
}

}  // namespace cute

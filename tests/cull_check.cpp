// Host check of the counting kernel's neighbour cull (count_impl.cuh:
// cull_keep2, with the radii of plan.cpp: cull_params).  The kernel drops a
// neighbour row when its FP32 gap to the bounding box of the item's home
// objects exceeds the reach; the box is taken over the homes' FP32 image
// coordinates x_i - S.  This replays that arithmetic with IEEE FP32
// operations (the same order, fused where the kernel fuses; the kernel's
// -(q - lo) is lo - q exactly) on pairs placed
// at and just inside the reach -- along the axes and the diagonals (where
// the per-axis rounding adds up most), near the far corners of large
// frames, across periodic images -- and requires every pair whose canonical
// FP64 separation (Sec. 2.2; sigma, pi: Sec. 3.4) is within the reach to be
// kept.  It also requires the cull to work: where the frame's rounding is
// small beside the reach, rows whose gap is 1e-4 beyond it are dropped.
// Prints "scenario pairs kept dropped violations"; exits 1 on a violation.
// With the argument "nomargin" the radii lose their widening: pairs at the
// reach are then dropped, and the check must say so.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -I include -I <csrc>
//        -I <cuda>/include cull_check.cpp <csrc>/plan.cpp -L<cuda>/lib64 -lcudart
#include "cute_internal.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

using namespace cute;

static float fsub(float a, float b) { volatile float r = a - b; return r; }
static float fmul(float a, float b) { volatile float r = a * b; return r; }
static float ffma(float a, float b, float c) { return std::fma(a, b, c); }

struct Scenario {
  const char *name;
  int kind;        // CUTE_MONO / CUTE_SIGMA_PI
  bool periodic;
  double L;        // periodic box
  double xm;       // frame half-extent (open)
  double r0, r1;   // reach (sigma, pi for CUTE_SIGMA_PI)
  double spread;   // extent of a home chunk
  bool tight;      // frame small enough that the radius stays within 1e-4 of the reach
};

static std::mt19937_64 rng(18331);
static bool g_nomargin = false;
static double U(double a, double b) { return std::uniform_real_distribution<double>(a, b)(rng); }

struct Result {
  long kept = 0, dropped = 0, violations = 0, beyond = 0, beyond_kept = 0;
};

static void run(const Scenario &sc, Result &res) {
  Geometry g;
  g.periodic = sc.periodic;
  g.L = sc.periodic ? sc.L : 0.0;
  for (int k = 0; k < 3; k++) g.xmax[k] = sc.periodic ? 0.5 * sc.L : sc.xm;
  DescInfo di;
  di.kind = sc.kind;
  di.g = &g;
  double e0[2] = {0.0, sc.r0}, e1[2] = {0.0, sc.r1};
  cute_pair_desc d;
  std::memset(&d, 0, sizeof(d));
  d.kind = (cute_kind)sc.kind;
  d.n0 = 1;
  d.edges0 = e0;
  d.n1 = 1;
  d.edges1 = sc.kind == CUTE_SIGMA_PI ? e1 : nullptr;
  KParams p;
  std::memset(&p, 0, sizeof(p));
  cull_params(std::vector<DescInfo>{di}, &d, 1, p);
  if (g_nomargin) {  // the radii without their widening (the check must then fail)
    p.cull_r2 = (float)(sc.r0 * sc.r0);
    p.cull_pi = (float)sc.r1;
  }
  const double half = sc.periodic ? 0.5 * sc.L : sc.xm;
  const float L32 = (float)sc.L;
  for (int trial = 0; trial < 20000; trial++) {
    // a home chunk of 1..64 objects (frame offsets, FP64) near a random
    // place -- often a far corner of the frame
    const int nh = trial % 3 == 0 ? 1 : 1 + (int)(rng() % 64);
    double c[3];
    for (int k = 0; k < 3; k++) {
      const double t = trial % 4 == 0 ? (U(0, 1) < 0.5 ? -1.0 : 1.0) * U(0.97, 1.0) : U(-1, 1);
      c[k] = t * (half - sc.spread);
    }
    std::vector<double> H(3 * nh);
    for (int i = 0; i < nh; i++)
      for (int k = 0; k < 3; k++) H[3 * i + k] = c[k] + (i ? U(-sc.spread, sc.spread) : 0.0);
    // image shift of the neighbour rows (periodic): S in {0, +L, -L} per axis
    int sh[3] = {0, 0, 0};
    if (sc.periodic)
      for (int k = 0; k < 3; k++) {
        if (H[k] > half - sc.r0 && U(0, 1) < 0.7) sh[k] = 1;        // neighbour past +L/2
        else if (H[k] < -half + sc.r0 && U(0, 1) < 0.7) sh[k] = -1;
      }
    // the kernel's box: FP32 offsets of the homes, minus the FP32 shift
    float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
    for (int i = 0; i < nh; i++)
      for (int k = 0; k < 3; k++) {
        const float a = (float)H[3 * i + k];
        const float S = sh[k] == 1 ? L32 : (sh[k] == -1 ? -L32 : 0.0f);
        const float x = fsub(a, S);
        lo[k] = std::min(lo[k], x);
        hi[k] = std::max(hi[k], x);
      }
    // neighbours of home 0 at the reach and just inside it
    for (int j = 0; j < 16; j++) {
      double u[3];
      const int dir = j % 4;
      if (dir == 0) {  // a diagonal
        for (int k = 0; k < 3; k++) u[k] = (rng() & 1) ? 1.0 : -1.0;
      } else if (dir == 1) {  // an axis
        for (int k = 0; k < 3; k++) u[k] = 0.0;
        u[rng() % 3] = (rng() & 1) ? 1.0 : -1.0;
      } else {
        for (int k = 0; k < 3; k++) u[k] = U(-1, 1);
      }
      double dvec[3];
      if (sc.kind == CUTE_SIGMA_PI) {
        // sigma at the reach in x-y and |pi| up to its reach (or the reverse)
        const double nxy = std::hypot(u[0], u[1]) + 1e-300;
        const double s = (j & 8) ? sc.r0 * U(0.999, 1.0) : sc.r0;
        const double pz = (j & 4) ? sc.r1 : sc.r1 * U(0.0, 1.0);
        dvec[0] = s * u[0] / nxy;
        dvec[1] = s * u[1] / nxy;
        dvec[2] = (u[2] < 0 ? -1.0 : 1.0) * pz;
      } else {
        const double n = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        const double s = (j & 8) ? sc.r0 * U(0.999, 1.0) : sc.r0;
        for (int k = 0; k < 3; k++) dvec[k] = s * u[k] / n;
      }
      // the neighbour's frame offset: home 0 + d, wrapped into the box when
      // it falls outside (its image is then home 0's shifted copy)
      double q[3];
      bool ok = true;
      for (int k = 0; k < 3; k++) {
        q[k] = H[k] - (sh[k] == 1 ? sc.L : (sh[k] == -1 ? -sc.L : 0.0)) + dvec[k];
        if (q[k] < -half || q[k] >= half) ok = false;  // outside the frame: not a catalog object
      }
      if (!ok) continue;
      // canonical FP64 separation from home 0 (its image)
      double s2 = 0.0, sxy = 0.0, pz = 0.0;
      for (int k = 0; k < 3; k++) {
        const double dk = q[k] - (H[k] - (sh[k] == 1 ? sc.L : (sh[k] == -1 ? -sc.L : 0.0)));
        s2 += dk * dk;
        if (k < 2) sxy += dk * dk;
        else pz = std::fabs(dk);
      }
      const bool within = sc.kind == CUTE_SIGMA_PI ? (sxy <= sc.r0 * sc.r0 && pz <= sc.r1)
                                                   : s2 <= sc.r0 * sc.r0;
      if (!within) continue;
      // the kernel's test
      float gq[3];
      for (int k = 0; k < 3; k++) {
        const float qf = (float)q[k];
        gq[k] = std::max(std::max(fsub(lo[k], qf), fsub(qf, hi[k])), 0.0f);
      }
      bool keep;
      if (sc.kind == CUTE_SIGMA_PI)
        keep = ffma(gq[1], gq[1], fmul(gq[0], gq[0])) <= p.cull_r2 && gq[2] <= p.cull_pi;
      else
        keep = ffma(gq[2], gq[2], ffma(gq[1], gq[1], fmul(gq[0], gq[0]))) <= p.cull_r2;
      if (keep) res.kept++;
      else {
        res.dropped++;
        res.violations++;
      }
    }
    // rows whose gap to the box is 1e-4 beyond the reach: dropped
    if (sc.tight) {
      double u[3] = {U(-1, 1), U(-1, 1), U(-1, 1)};
      const double n = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      float gq[3];
      const double gap = (sc.kind == CUTE_SIGMA_PI ? sc.r0 : sc.r0) * (1.0 + 1e-4);
      for (int k = 0; k < 3; k++) gq[k] = (float)std::fabs(gap * u[k] / n);
      if (sc.kind == CUTE_SIGMA_PI) {
        const double nxy = std::hypot(u[0], u[1]) + 1e-300;
        gq[0] = (float)std::fabs(gap * u[0] / nxy);
        gq[1] = (float)std::fabs(gap * u[1] / nxy);
        gq[2] = 0.0f;
      }
      bool keep;
      if (sc.kind == CUTE_SIGMA_PI)
        keep = ffma(gq[1], gq[1], fmul(gq[0], gq[0])) <= p.cull_r2 && gq[2] <= p.cull_pi;
      else
        keep = ffma(gq[2], gq[2], ffma(gq[1], gq[1], fmul(gq[0], gq[0]))) <= p.cull_r2;
      res.beyond++;
      if (keep) res.beyond_kept++;
    }
  }
}

int main(int argc, char **argv) {
  g_nomargin = argc > 1 && std::strcmp(argv[1], "nomargin") == 0;
  const Scenario sc[] = {
      {"mono_open_small", CUTE_MONO, false, 0, 1000.0, 200.0, 0, 30.0, true},
      {"mono_open_far", CUTE_MONO, false, 0, 1.0e6, 200.0, 0, 30.0, false},
      {"mono_open_extreme", CUTE_MONO, false, 0, 9.0e7, 150.0, 0, 10.0, false},
      {"chord_unit", CUTE_MONO, false, 0, 1.0, 0.1743114854953163, 0, 0.002, true},
      {"mono_periodic", CUTE_MONO, true, 2000.0, 0, 150.0, 0, 20.0, true},
      {"mono_periodic_big", CUTE_MONO, true, 1.0e6, 0, 300.0, 0, 40.0, false},
      {"sigpi_periodic", CUTE_SIGMA_PI, true, 1500.0, 0, 150.0, 150.0, 20.0, true},
      {"sigpi_periodic_flat", CUTE_SIGMA_PI, true, 1500.0, 0, 50.0, 200.0, 20.0, true},
      {"sigpi_open", CUTE_SIGMA_PI, false, 0, 3000.0, 100.0, 40.0, 10.0, true},
  };
  int bad = 0;
  for (const Scenario &s : sc) {
    Result r;
    run(s, r);
    std::printf("%s %ld %ld %ld beyond %ld kept %ld\n", s.name, r.kept, r.dropped, r.violations,
                r.beyond, r.beyond_kept);
    if (r.violations || r.kept < 1000 || r.beyond_kept) bad = 1;
  }
  return bad;
}

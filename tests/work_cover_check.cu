// Host check of the counting kernels' work decomposition (Sec. 3.3 cell
// lists; the chunk/stencil/segment form of plan.cpp and count_kernel.cuh):
// objects are placed in a cell grid that follows the grid contract (cells
// no smaller than reach / k on each axis, x cut 8 times finer, a periodic
// axis at least 2k + 1 cells), the home chunks (chunks_build), the stencil
// rows (stencil_build) and every entry's segments (entry_segments) are
// expanded into the object pairs they hand to the kernel -- their number
// must equal the work builder's count of them (work_pairs.h: segment_pairs,
// the stencil_pairs statistic) -- and each pair's multiplicity is checked: every pair within reach exactly once -- unordered
// pairs for the half stencil of an auto count, ordered pairs i != j for the
// full stencil (the adjoint), every (a, b) for a cross count -- and with the
// periodic image the segment gives it (the kernel's separation
// x_j - x_i + S, S = +L or -L per axis from the segment's shift code) within
// reach.  A pair beyond reach may be met twice on a periodic row (a wide
// home chunk's x-range and the wrapped range of a chunk at the row's end):
// beyond reach under the minimum image it is beyond reach under every
// image, out of range both times, so those are counted and reported, not
// failed.  Host code only (compiled by nvcc because the segment function
// lives in a header that also holds device code).
// Prints "scenario pairs_enumerated pairs_in_reach duplicates_beyond_reach
// violations"; exits 1 on any violation.
#include "count_kernel.cuh"
#include "work_pairs.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

using namespace cute;

struct Cat {
  std::vector<double> x;   // n x 3, in cell order
  std::vector<int32_t> cs; // cell_start, ncell + 1
};

// the smallest k >= kreq whose cells (no smaller than reach / k) still
// leave 2k + 1 of them on a periodic axis; the open axis takes kreq
static void make_geometry(Geometry &g, bool periodic, double L, const double lo[3],
                          const double hi[3], const double reach[3], int kreq) {
  g.periodic = periodic;
  g.L = L;
  for (int d = 0; d < 3; d++) {
    const int kr = d == 0 ? 8 * kreq : kreq;
    if (periodic) {
      int k = kr;
      long long n = (long long)std::floor(L / (reach[d] * (1 + 1e-9) / k));
      while (n < 2 * k + 1) {
        k++;
        n = (long long)std::floor(L / (reach[d] * (1 + 1e-9) / k));
      }
      g.nc[d] = (int)n;
      g.a[d] = L / n;
      g.k[d] = (int)std::ceil(reach[d] * (1 + 1e-9) / g.a[d]);
      g.origin[d] = 0;
    } else {
      const double amin = reach[d] * (1 + 1e-9) / kr, ext = hi[d] - lo[d];
      const long long n = (long long)std::floor(ext / amin) + 1;
      g.nc[d] = (int)n;
      g.a[d] = std::max(amin, ext / n * (1 + 1e-12));
      g.k[d] = (int)std::max(1.0, std::ceil(reach[d] * (1 + 1e-9) / g.a[d]));
      g.origin[d] = lo[d];
    }
  }
}

static Cat place(const Geometry &g, const std::vector<double> &pts) {
  const int n = (int)pts.size() / 3;
  const long long ncell = (long long)g.nc[0] * g.nc[1] * g.nc[2];
  std::vector<long long> cid(n);
  Cat c;
  c.cs.assign(ncell + 1, 0);
  for (int i = 0; i < n; i++) {
    int q[3];
    for (int d = 0; d < 3; d++) {
      const double f = std::floor((pts[3 * i + d] - g.origin[d]) / g.a[d]);
      q[d] = (int)std::min<double>(std::max<double>(f, 0.0), g.nc[d] - 1);
    }
    cid[i] = ((long long)q[2] * g.nc[1] + q[1]) * g.nc[0] + q[0];
    c.cs[cid[i] + 1]++;
  }
  for (long long k = 0; k < ncell; k++) c.cs[k + 1] += c.cs[k];
  std::vector<int> order(n);
  for (int i = 0; i < n; i++) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cid[a] < cid[b]; });
  c.x.resize(pts.size());
  for (int i = 0; i < n; i++)
    for (int d = 0; d < 3; d++) c.x[3 * i + d] = pts[3 * order[i] + d];
  return c;
}

// uniform objects, and every third group of 20 in a Gaussian clump (many
// objects per cell: chunks that straddle cells, runs cut at home_chunk)
static std::vector<double> objects(std::mt19937_64 &g, int n, const double lo[3], const double hi[3],
                                   double blob) {
  std::uniform_real_distribution<double> U(0, 1);
  std::normal_distribution<double> N(0, 1);
  std::vector<double> p(3 * n);
  double c[3] = {0, 0, 0};
  for (int i = 0; i < n; i++) {
    if (i % 20 == 0)
      for (int d = 0; d < 3; d++) c[d] = lo[d] + (hi[d] - lo[d]) * U(g);
    const bool clump = (i / 20) % 3 == 0;
    for (int d = 0; d < 3; d++) {
      const double w = hi[d] - lo[d];
      double v = clump ? c[d] + blob * N(g) : lo[d] + w * U(g);
      v = lo[d] + std::fmod(std::fmod(v - lo[d], w) + w, w);
      if (v >= hi[d]) v = lo[d];
      p[3 * i + d] = v;
    }
  }
  return p;
}

// separation d within the region stencil_build is built for (ball, disk x
// slab, box)
static bool within(const double d[3], int shape, const double need[3]) {
  if (shape == kShapeBall) return d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < need[0] * need[0];
  if (shape == kShapeDiskSlab)
    return d[0] * d[0] + d[1] * d[1] < need[0] * need[0] && std::fabs(d[2]) < need[2];
  return std::fabs(d[0]) < need[0] && std::fabs(d[1]) < need[1] && std::fabs(d[2]) < need[2];
}

// within reach under the minimum image
static bool in_reach(const double *a, const double *b, bool periodic, double L, int shape,
                     const double need[3]) {
  double d[3];
  for (int k = 0; k < 3; k++) {
    d[k] = b[k] - a[k];
    if (periodic) {
      if (d[k] > 0.5 * L) d[k] -= L;
      else if (d[k] < -0.5 * L) d[k] += L;
    }
  }
  return within(d, shape, need);
}

// mode: kModeAutoHalf, kModeAutoFull or kModeCross
static long run(const char *name, bool periodic, double L, const double lo[3], const double hi[3],
                const double need[3], int shape, int kreq, int home_chunk, int mode, int na, int nb,
                double blob, std::mt19937_64 &rng) {
  Geometry g;
  make_geometry(g, periodic, L, lo, hi, need, kreq);
  const Cat A = place(g, objects(rng, na, lo, hi, blob));
  const Cat B = mode == kModeCross ? place(g, objects(rng, nb, lo, hi, blob)) : A;
  const int nA = (int)A.x.size() / 3, nB = (int)B.x.size() / 3;
  std::vector<int4> chunks, stencil;
  chunks_build(g, A.cs.data(), home_chunk, chunks);
  stencil_build(g, mode != kModeCross, mode == kModeAutoFull, shape, need, stencil);
  PairWork pd;
  std::memset(&pd, 0, sizeof pd);
  pd.chunks = chunks.data();
  pd.stencil = stencil.data();
  pd.csB = B.cs.data();
  pd.nchunks = (int)chunks.size();
  pd.nstencil = (int)stencil.size();
  pd.nx = g.nc[0];
  pd.ny = g.nc[1];
  pd.nz = g.nc[2];
  pd.mode = mode;
  pd.periodic = periodic;
  std::vector<unsigned char> mult((size_t)nA * nB, 0), hit((size_t)nA * nB, 0);
  long enumerated = 0, bad = 0, dup = 0;
  unsigned long long presented = 0;  // the work builder's count of the same pairs
  for (const int4 &c : chunks) {
    if (c.y - c.x > home_chunk) bad++;
    for (const int4 &r : stencil) {
      Seg s[3];
      const int ns = entry_segments(pd, pd.csB, c, r, s);
      for (int k = 0; k < ns; k++) {
        presented += segment_pairs(c, s[k]);
        const int code = (s[k].flags >> 8) & 63;
        double S[3];
        for (int a = 0; a < 3; a++) {
          const int q = (code >> (2 * a)) & 3;
          S[a] = q == 1 ? L : (q == 2 ? -L : 0.0);
        }
        for (int i = c.x; i < c.y; i++)
          for (int j = s[k].j0; j < s[k].j1; j++) {
            if ((s[k].flags & kSegSelf) && j <= i) continue;
            if ((s[k].flags & kSegNoSelfPair) && j == i) continue;
            if (mode != kModeCross && i == j) { bad++; continue; }
            size_t key = (size_t)i * nB + j;
            if (mode == kModeAutoHalf) key = (size_t)std::min(i, j) * nB + std::max(i, j);
            if (mult[key] < 255) mult[key]++;
            double d[3];
            for (int a = 0; a < 3; a++) d[a] = B.x[3 * j + a] - A.x[3 * i + a] + S[a];
            if (within(d, shape, need)) hit[key] = 1;
            enumerated++;
          }
      }
    }
  }
  if (presented != (unsigned long long)enumerated) {
    std::printf("  stencil pairs %llu, enumerated %ld\n", presented, enumerated);
    bad++;
  }
  long inreach = 0;
  for (int i = 0; i < nA; i++)
    for (int j = 0; j < nB; j++) {
      if (mode != kModeCross && (i == j || (mode == kModeAutoHalf && j < i))) continue;
      const size_t key = (size_t)i * nB + j;
      const unsigned m = mult[key];
      const bool want = in_reach(&A.x[3 * i], &B.x[3 * j], periodic, L, shape, need);
      inreach += want;
      if (!want) {
        dup += m > 1;
        if (hit[key]) bad++;  // beyond reach, yet some image within it
        continue;
      }
      if (m != 1 || !hit[key]) {
        if (bad < 5)
          std::printf("  pair (%d, %d): met %u times, image within reach %d\n", i, j, m, hit[key]);
        bad++;
      }
    }
  std::printf("%s %ld %ld %ld %ld\n", name, enumerated, inreach, dup, bad);
  return bad;
}

int main() {
  std::mt19937_64 rng(20121008);
  long bad = 0;
  const double z0[3] = {0, 0, 0};
  const double box100[3] = {100, 100, 100}, box30[3] = {30, 30, 30};
  const double olo[3] = {-120, 300, 40}, ohi[3] = {80, 420, 160};
  const double r12[3] = {12, 12, 12}, r13[3] = {13, 13, 13}, r3[3] = {3, 3, 3};
  const double sp[3] = {15, 15, 9};
  const int modes[3] = {kModeAutoHalf, kModeAutoFull, kModeCross};
  const char *mn[3] = {"auto_half", "auto_full", "cross"};
  for (int m = 0; m < 3; m++) {
    for (int hc : {64, 128}) {
      std::string t = std::string(mn[m]) + "_hc" + std::to_string(hc);
      bad += run(("periodic_ball_" + t).c_str(), true, 100, z0, box100, r12, kShapeBall, 2, hc,
                 modes[m], 1800, 1100, 1.5, rng);
      bad += run(("periodic_small_box_" + t).c_str(), true, 30, z0, box30, r13, kShapeBall, 2, hc,
                 modes[m], 700, 500, 1.0, rng);
      bad += run(("periodic_diskslab_" + t).c_str(), true, 100, z0, box100, sp, kShapeDiskSlab, 3,
                 hc, modes[m], 1500, 900, 2.0, rng);
      bad += run(("periodic_fine_grid_" + t).c_str(), true, 100, z0, box100, r3, kShapeBall, 2, hc,
                 modes[m], 2500, 1500, 0.3, rng);
      bad += run(("open_ball_" + t).c_str(), false, 0, olo, ohi, r12, kShapeBall, 1, hc, modes[m],
                 1800, 1100, 1.5, rng);
      bad += run(("open_box_" + t).c_str(), false, 0, olo, ohi, r12, kShapeBox, 3, hc, modes[m],
                 1500, 900, 1.5, rng);
      bad += run(("open_diskslab_" + t).c_str(), false, 0, olo, ohi, sp, kShapeDiskSlab, 2, hc,
                 modes[m], 1500, 900, 2.0, rng);
    }
  }
  // finer grids: 4 to 8 cells per reach (the range cute_grid_build accepts
  // above the defaults, and where warm-up tuning may take a count)
  for (int k = 4; k <= 8; k++)
    for (int m = 0; m < 3; m++)
      for (int hc : {64, 128}) {
        std::string t = std::string(mn[m]) + "_hc" + std::to_string(hc) + "_k" + std::to_string(k);
        bad += run(("periodic_ball_" + t).c_str(), true, 100, z0, box100, r12, kShapeBall, k, hc,
                   modes[m], 1800, 1100, 1.5, rng);
        bad += run(("periodic_diskslab_" + t).c_str(), true, 100, z0, box100, sp, kShapeDiskSlab,
                   k, hc, modes[m], 1500, 900, 2.0, rng);
        bad += run(("open_ball_" + t).c_str(), false, 0, olo, ohi, r12, kShapeBall, k, hc,
                   modes[m], 1800, 1100, 1.5, rng);
        bad += run(("open_box_" + t).c_str(), false, 0, olo, ohi, r12, kShapeBox, k, hc,
                   modes[m], 1500, 900, 1.5, rng);
        bad += run(("open_diskslab_" + t).c_str(), false, 0, olo, ohi, sp, kShapeDiskSlab, k, hc,
                   modes[m], 1500, 900, 2.0, rng);
      }
  return bad ? 1 : 0;
}

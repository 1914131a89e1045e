// Host check of the double-float re-test stage (paper_1210_1833_gb300/
// csrc/df_stage.h): on pairs placed on, and a hair off, every edge, every
// slot the stage decides must be the slot of the canonical FP64 formulas
// (Sec. 2.2: d^2, sigma^2 and pi^2 against squared edges with the minimum
// image; Sec. 3.4: mu about the midpoint line of sight, q >= m_k^2 r^2 l^2).
// Prints "cases decided mismatches" per scenario; exits 1 on any mismatch.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off df_stage_check.cpp
#include "../paper_1210_1833_gb300/csrc/df_stage.h"

#include <cstdio>
#include <random>
#include <vector>

using namespace cute;

struct Frame {
  double fo[3];  // FP32 frame centre
  double xm;     // largest |x - fo|
  double L;      // periodic box, 0 open
};

// the grid's FP32 offset and remainder of one coordinate
static void split(double x, double fo, float &p, float &lo) {
  const double o = x - fo;
  p = (float)o;
  lo = (float)(o - (double)p);
}

static double wrap(double d, double L) {
  if (L > 0) {
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
  }
  return d;
}
// canonical bin of v on squared edges E (n bins): -1 outside
static int bin64(const std::vector<double> &E, double v) {
  const int n = (int)E.size() - 1;
  if (!(v >= E[0]) || !(v < E[n])) return -1;
  int b = 0;
  while (b + 1 <= n && v >= E[b + 1]) b++;
  return b;
}

static std::vector<double> sq_edges(double step, int n) {
  std::vector<double> E(n + 1);
  for (int k = 0; k <= n; k++) E[k] = (k * step) * (k * step);
  return E;
}
static std::vector<float> split_edges(const std::vector<double> &E) {
  std::vector<float> o(2 * E.size());
  for (size_t k = 0; k < E.size(); k++) {
    o[2 * k] = (float)E[k];
    o[2 * k + 1] = (float)(E[k] - (double)o[2 * k]);
  }
  return o;
}

struct Tally {
  long cases = 0, decided = 0, bad = 0;
  void add(int df, int canon) {
    cases++;
    if (df == -2) return;
    decided++;
    if (df != canon) {
      if (bad < 5) std::printf("  mismatch: stage %d canonical %d\n", df, canon);
      bad++;
    }
  }
};

// relative offsets from an edge: exact, below, around and above the stage's margin
static const double kOff[] = {0.0,    1e-13, -1e-13, 1e-11, -1e-11, 3e-11, -3e-11, 1e-10,
                              -1e-10, 1e-9,  -1e-9,  1e-7,  -1e-7,  1e-4,  -1e-4,  0.3};

static void unit(std::mt19937_64 &g, double *u) {
  std::normal_distribution<double> N(0, 1);
  double n2 = 0;
  for (int k = 0; k < 3; k++) {
    u[k] = N(g);
    n2 += u[k] * u[k];
  }
  const double n = std::sqrt(n2);
  for (int k = 0; k < 3; k++) u[k] /= n;
}

// monopole pairs around every edge; periodic pairs straddle the faces
static Tally run_mono(const Frame &F, double step, int n, double spread, bool chord,
                      std::mt19937_64 &g) {
  const std::vector<double> E = sq_edges(step, n);
  const std::vector<float> Ed = split_edges(E);
  const float inv = (float)(1.0 / step);
  const float eta = (float)dfs::eta_sep(F.xm, F.L);
  const float Lh = (float)F.L, Ll = (float)(F.L - (double)Lh);
  std::uniform_real_distribution<double> U(-1, 1);
  Tally t;
  for (int k = 1; k <= n; k++)
    for (double off : kOff)
      for (int rep = 0; rep < 40; rep++) {
        double a[3], b[3], u[3];
        unit(g, u);
        const double e = k * step * (1.0 + off);
        for (int c = 0; c < 3; c++) {
          if (chord) {
            a[c] = 0;  // filled below
          } else if (F.L > 0) {
            a[c] = std::fmod(F.fo[c] + spread * U(g) + 10 * F.L, F.L);
          } else {
            a[c] = F.fo[c] + spread * U(g);
          }
        }
        if (chord) {
          double v[3];
          unit(g, v);
          for (int c = 0; c < 3; c++) a[c] = v[c];
          double t2[3];
          unit(g, t2);
          double dot = t2[0] * v[0] + t2[1] * v[1] + t2[2] * v[2];
          double tn = 0;
          for (int c = 0; c < 3; c++) {
            t2[c] -= dot * v[c];
            tn += t2[c] * t2[c];
          }
          tn = std::sqrt(tn);
          const double ang = 2 * std::asin(std::min(1.0, e / 2));
          for (int c = 0; c < 3; c++) b[c] = std::cos(ang) * v[c] + std::sin(ang) * t2[c] / tn;
        } else {
          for (int c = 0; c < 3; c++) {
            b[c] = a[c] + u[c] * e;
            if (F.L > 0) {
              b[c] = std::fmod(b[c] + 10 * F.L, F.L);
              if (b[c] >= F.L) b[c] = 0;
            }
          }
        }
        float pa[3], la[3], pb[3], lb[3];
        double d2 = 0;
        double dd[3];
        for (int c = 0; c < 3; c++) {
          split(a[c], F.fo[c], pa[c], la[c]);
          split(b[c], F.fo[c], pb[c], lb[c]);
          dd[c] = wrap(b[c] - a[c], F.L);
        }
        d2 = (dd[0] * dd[0] + dd[1] * dd[1]) + dd[2] * dd[2];
        const int cb = bin64(E, d2);
        const int canon = cb < 0 ? 0 : cb + 1;
        t.add(dfs::mono_slot(pa, la, pb, lb, eta, Lh, Ll, inv, Ed.data(), n), canon);
      }
  return t;
}

static Tally run_sigpi(const Frame &F, double s0, int n0, double s1, int n1, double spread,
                       std::mt19937_64 &g) {
  const std::vector<double> E0 = sq_edges(s0, n0), E1 = sq_edges(s1, n1);
  const std::vector<float> E0d = split_edges(E0), E1d = split_edges(E1);
  const float eta = (float)dfs::eta_sep(F.xm, F.L);
  const float Lh = (float)F.L, Ll = (float)(F.L - (double)Lh);
  std::uniform_real_distribution<double> U(-1, 1), U01(0, 1);
  Tally t;
  for (int axis = 0; axis < 2; axis++) {
    const int n = axis ? n1 : n0;
    const double st = axis ? s1 : s0;
    for (int k = 1; k <= n; k++)
      for (double off : kOff)
        for (int rep = 0; rep < 30; rep++) {
          const double e = k * st * (1.0 + off);
          double sig = axis ? U01(g) * s0 * n0 : e;
          double pi = axis ? e : U01(g) * s1 * n1;
          const double phi = 6.283185307179586 * U01(g);
          const double off3[3] = {sig * std::cos(phi), sig * std::sin(phi), U(g) > 0 ? pi : -pi};
          double a[3], b[3];
          for (int c = 0; c < 3; c++) {
            a[c] = F.L > 0 ? std::fmod(F.fo[c] + spread * U(g) + 10 * F.L, F.L)
                           : F.fo[c] + spread * U(g);
            b[c] = a[c] + off3[c];
            if (F.L > 0) {
              b[c] = std::fmod(b[c] + 10 * F.L, F.L);
              if (b[c] >= F.L) b[c] = 0;
            }
          }
          float pa[3], la[3], pb[3], lb[3];
          double dd[3];
          for (int c = 0; c < 3; c++) {
            split(a[c], F.fo[c], pa[c], la[c]);
            split(b[c], F.fo[c], pb[c], lb[c]);
            dd[c] = wrap(b[c] - a[c], F.L);
          }
          const int bs = bin64(E0, dd[0] * dd[0] + dd[1] * dd[1]);
          const int bp = bin64(E1, dd[2] * dd[2]);
          const int canon = (bs < 0 || bp < 0) ? 0 : (bs + 1) * (n1 + 2) + bp + 1;
          t.add(dfs::sigpi_slot(pa, la, pb, lb, eta, Lh, Ll, (float)(1.0 / s0), E0d.data(), n0,
                                (float)(1.0 / s1), E1d.data(), n1),
                canon);
        }
  }
  return t;
}

// (r, mu): observer at the origin, objects at distances around dist
static Tally run_rmu(double dist, const double *fo, double xm, double am, double s0, int n0,
                     int n1, std::mt19937_64 &g) {
  const std::vector<double> E0 = sq_edges(s0, n0);
  std::vector<double> M(n1 + 1);
  for (int k = 0; k <= n1; k++) M[k] = ((double)k / n1) * ((double)k / n1);
  const std::vector<float> E0d = split_edges(E0), Md = split_edges(M);
  double fom = std::max(std::fabs(fo[0]), std::max(std::fabs(fo[1]), std::fabs(fo[2])));
  const float eta = (float)dfs::eta_sep(xm, 0.0), eta_l = (float)dfs::eta_los(xm, fom, am);
  float fo2h[3], fo2l[3];
  for (int c = 0; c < 3; c++) {
    fo2h[c] = (float)(2 * fo[c]);
    fo2l[c] = (float)(2 * fo[c] - (double)fo2h[c]);
  }
  Tally t;
  const double rs[] = {0.3, 0.7, 3.0, 12.0, 77.0, 150.0, 199.0};
  for (double r : rs)
    for (int k = 0; k <= n1; k++)
      for (double off : kOff)
        for (int rep = 0; rep < 6; rep++) {
          double xi[3], tt[3];
          unit(g, xi);
          for (int c = 0; c < 3; c++) xi[c] = fo[c] + (xi[c] * dist * 0.3);
          unit(g, tt);
          const double mm = std::min(std::max((double)k / n1 * (1.0 + off), 0.0), 1.0);
          double s[3] = {0, 0, 0};
          for (int it = 0; it < 8; it++) {  // direction relative to l = 2 x_i + s
            double l[3], ln = 0;
            for (int c = 0; c < 3; c++) {
              l[c] = 2 * xi[c] + s[c];
              ln += l[c] * l[c];
            }
            ln = std::sqrt(ln);
            double dot = 0;
            for (int c = 0; c < 3; c++) dot += tt[c] * l[c] / ln;
            double tp[3], tn = 0;
            for (int c = 0; c < 3; c++) {
              tp[c] = tt[c] - dot * l[c] / ln;
              tn += tp[c] * tp[c];
            }
            tn = std::sqrt(tn);
            for (int c = 0; c < 3; c++)
              s[c] = r * (mm * l[c] / ln + std::sqrt(std::max(0.0, 1 - mm * mm)) * tp[c] / tn);
          }
          double xj[3];
          for (int c = 0; c < 3; c++) xj[c] = xi[c] + s[c];
          // canonical (Sec. 3.4 reading): s = x_j - x_i, l = x_i + x_j
          double sx = xj[0] - xi[0], sy = xj[1] - xi[1], sz = xj[2] - xi[2];
          double lx = xi[0] + xj[0], ly = xi[1] + xj[1], lz = xi[2] + xj[2];
          double r2 = (sx * sx + sy * sy) + sz * sz;
          int canon = 0;
          const int br = bin64(E0, r2);
          if (br >= 0) {
            int bm = 0;
            if (r2 != 0.0) {
              double l2 = (lx * lx + ly * ly) + lz * lz;
              double sl = (sx * lx + sy * ly) + sz * lz;
              double q = sl * sl, den = r2 * l2;
              for (int m = 1; m <= n1 - 1; m++)
                if (q >= M[m] * den) bm = m;
            }
            canon = (br + 1) * (n1 + 2) + bm + 1;
          }
          float pa[3], la[3], pb[3], lb[3];
          for (int c = 0; c < 3; c++) {
            split(xi[c], fo[c], pa[c], la[c]);
            split(xj[c], fo[c], pb[c], lb[c]);
          }
          t.add(dfs::rmu_slot(pa, la, pb, lb, eta, eta_l, fo2h, fo2l, (float)(1.0 / s0),
                              E0d.data(), n0, (float)n1, Md.data(), n1),
                canon);
        }
  return t;
}

// ---- integer lattices: integer coordinates and edges make every FP64
// quantity of the canonical formulas exact, so many pairs sit exactly on an
// edge; the stage must leave those to FP64 or decide them exactly right.
// Every pair of the points is checked; `ties` counts the exact ties.
static std::vector<double> lattice(std::mt19937_64 &g, int n, const double lo[3], const double hi[3]) {
  std::vector<double> p(3 * n);
  for (int i = 0; i < n; i++)
    for (int c = 0; c < 3; c++) {
      std::uniform_int_distribution<int> U((int)lo[c], (int)hi[c] - 1);
      p[3 * i + c] = U(g);
    }
  return p;
}

static Tally run_lattice_mono_sigpi(const Frame &F, bool sigpi, int n0, int n1,
                                    const std::vector<double> &x, long &ties) {
  const std::vector<double> E0 = sq_edges(1.0, n0), E1 = sq_edges(1.0, n1);
  const std::vector<float> E0d = split_edges(E0), E1d = split_edges(E1);
  const float eta = (float)dfs::eta_sep(F.xm, F.L);
  const float Lh = (float)F.L, Ll = (float)(F.L - (double)Lh);
  const int n = (int)x.size() / 3;
  Tally t;
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++) {
      float pa[3], la[3], pb[3], lb[3];
      double dd[3];
      for (int c = 0; c < 3; c++) {
        split(x[3 * i + c], F.fo[c], pa[c], la[c]);
        split(x[3 * j + c], F.fo[c], pb[c], lb[c]);
        dd[c] = wrap(x[3 * j + c] - x[3 * i + c], F.L);
      }
      if (!sigpi) {
        const double d2 = (dd[0] * dd[0] + dd[1] * dd[1]) + dd[2] * dd[2];
        const int cb = bin64(E0, d2);
        for (int k = 1; k <= n0; k++) ties += d2 == E0[k];
        t.add(dfs::mono_slot(pa, la, pb, lb, eta, Lh, Ll, 1.0f, E0d.data(), n0), cb < 0 ? 0 : cb + 1);
      } else {
        const double sg2 = dd[0] * dd[0] + dd[1] * dd[1], pi2 = dd[2] * dd[2];
        const int bs = bin64(E0, sg2), bp = bin64(E1, pi2);
        for (int k = 1; k <= n0; k++) ties += sg2 == E0[k];
        for (int k = 1; k <= n1; k++) ties += pi2 == E1[k];
        const int canon = (bs < 0 || bp < 0) ? 0 : (bs + 1) * (n1 + 2) + bp + 1;
        t.add(dfs::sigpi_slot(pa, la, pb, lb, eta, Lh, Ll, 1.0f, E0d.data(), n0, 1.0f, E1d.data(),
                              n1),
              canon);
      }
    }
  return t;
}

// (r, mu) on a lattice far from the observer, with pairs at exactly mu = 1/2:
// s = 2 m s0, l = x_i + x_j = 2 q (1, 1, 0), s0 at 60 degrees to (1, 1, 0)
static Tally run_lattice_rmu(std::mt19937_64 &g, long &ties) {
  const int n0 = 13, n1 = 4;
  std::vector<double> x;
  const int s0[4][3] = {{1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}};
  for (int q = 300; q < 340; q += 8)
    for (int m = 1; m <= 4; m++)
      for (auto &v : s0)
        for (int sg = -1; sg <= 1; sg += 2)
          for (int c = 0; c < 3; c++) x.push_back((c < 2 ? q : 0) + sg * m * v[c]);
  const double lo[3] = {300, 300, -10}, hi[3] = {341, 341, 11};
  const std::vector<double> r = lattice(g, 200, lo, hi);
  x.insert(x.end(), r.begin(), r.end());
  const double fo[3] = {320.25, 319.5, 0.125};
  double xm = 0, am = 0;
  for (size_t i = 0; i < x.size(); i += 3) {
    double a2 = 0;
    for (int c = 0; c < 3; c++) {
      xm = std::max(xm, std::fabs(x[i + c] - fo[c]));
      a2 += x[i + c] * x[i + c];
    }
    am = std::max(am, std::sqrt(a2));
  }
  const double fom = std::max(std::fabs(fo[0]), std::max(std::fabs(fo[1]), std::fabs(fo[2])));
  const std::vector<double> E0 = sq_edges(1.0, n0);
  std::vector<double> M(n1 + 1);
  for (int k = 0; k <= n1; k++) M[k] = ((double)k / n1) * ((double)k / n1);
  const std::vector<float> E0d = split_edges(E0), Md = split_edges(M);
  const float eta = (float)dfs::eta_sep(xm, 0.0), eta_l = (float)dfs::eta_los(xm, fom, am);
  float fo2h[3], fo2l[3];
  for (int c = 0; c < 3; c++) {
    fo2h[c] = (float)(2 * fo[c]);
    fo2l[c] = (float)(2 * fo[c] - (double)fo2h[c]);
  }
  const int n = (int)x.size() / 3;
  Tally t;
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++) {
      const double *xi = &x[3 * i], *xj = &x[3 * j];
      const double sx = xj[0] - xi[0], sy = xj[1] - xi[1], sz = xj[2] - xi[2];
      const double lx = xi[0] + xj[0], ly = xi[1] + xj[1], lz = xi[2] + xj[2];
      const double r2 = (sx * sx + sy * sy) + sz * sz;
      int canon = 0;
      const int br = bin64(E0, r2);
      for (int k = 1; k <= n0; k++) ties += r2 == E0[k];
      if (br >= 0) {
        int bm = 0;
        if (r2 != 0.0) {
          const double l2 = (lx * lx + ly * ly) + lz * lz;
          const double sl = (sx * lx + sy * ly) + sz * lz;
          const double qv = sl * sl, den = r2 * l2;
          for (int m = 1; m <= n1 - 1; m++) {
            if (qv >= M[m] * den) bm = m;
            ties += qv == M[m] * den;
          }
        }
        canon = (br + 1) * (n1 + 2) + bm + 1;
      }
      float pa[3], la[3], pb[3], lb[3];
      for (int c = 0; c < 3; c++) {
        split(xi[c], fo[c], pa[c], la[c]);
        split(xj[c], fo[c], pb[c], lb[c]);
      }
      t.add(dfs::rmu_slot(pa, la, pb, lb, eta, eta_l, fo2h, fo2l, 1.0f, E0d.data(), n0, (float)n1,
                          Md.data(), n1),
            canon);
    }
  return t;
}

int main() {
  std::mt19937_64 g(20121008);
  long bad = 0;
  auto report = [&](const char *name, const Tally &t) {
    std::printf("%s %ld %ld %ld\n", name, t.cases, t.decided, t.bad);
    bad += t.bad;
  };
  {
    Frame F{{1234.5, -300.25, 77.0}, 1500.0, 0.0};
    report("mono_open", run_mono(F, 2.5, 40, 1400.0, false, g));
  }
  {
    Frame F{{1000.0, 1000.0, 1000.0}, 1000.0, 2000.0};
    report("mono_periodic", run_mono(F, 5.0, 30, 1000.0, false, g));
  }
  {
    Frame F{{750.0, 750.0, 750.0}, 750.0, 1500.0 + 1.0 / 3.0};  // box not exact in FP32
    report("mono_periodic_odd_box", run_mono(F, 7.0, 20, 750.0, false, g));
  }
  {
    Frame F{{0.01, -0.02, 0.97}, 0.3, 0.0};
    report("chord", run_mono(F, 0.0027, 64, 0.0, true, g));
  }
  {
    Frame F{{750.0, 750.0, 750.0}, 750.0, 1500.0};
    report("sigpi_periodic", run_sigpi(F, 3.0, 50, 3.0, 50, 750.0, g));
  }
  {
    Frame F{{-5000.0, 20.0, 333.3}, 400.0, 0.0};
    report("sigpi_open", run_sigpi(F, 2.0, 15, 2.5, 10, 390.0, g));
  }
  {
    const double fo[3] = {1250.0, 1083.0, 625.0};
    report("rmu_lightcone", run_rmu(1700.0, fo, 0.3 * 1700.0 + 200.0, 1768.0 + 0.3 * 1700.0 + 200.0,
                                    5.0, 40, 40, g));
  }
  {
    const double fo[3] = {0.0, 0.0, 0.0};
    report("rmu_centred", run_rmu(1500.0, fo, 0.3 * 1500.0 + 200.0, 0.3 * 1500.0 + 200.0, 5.0, 40,
                                  40, g));
  }
  {
    // lattices: "name cases decided mismatches", then "name_ties count"
    long ties = 0;
    const double lo[3] = {0, 0, 0}, hi[3] = {40, 40, 40};
    const std::vector<double> xp = lattice(g, 320, lo, hi);
    Frame F{{20.0, 20.0, 20.0}, 20.0, 40.0};
    report("lattice_mono_periodic", run_lattice_mono_sigpi(F, false, 13, 1, xp, ties));
    std::printf("lattice_mono_periodic_ties %ld\n", ties);
    ties = 0;
    const double olo[3] = {985, -315, 62}, ohi[3] = {1016, -284, 93};
    Frame Fo{{1000.37, -299.81, 77.5}, 16.0, 0.0};
    report("lattice_mono_open", run_lattice_mono_sigpi(Fo, false, 13, 1, lattice(g, 320, olo, ohi),
                                                       ties));
    std::printf("lattice_mono_open_ties %ld\n", ties);
    ties = 0;
    report("lattice_sigpi_periodic", run_lattice_mono_sigpi(F, true, 9, 7, xp, ties));
    std::printf("lattice_sigpi_periodic_ties %ld\n", ties);
    ties = 0;
    report("lattice_rmu", run_lattice_rmu(g, ties));
    std::printf("lattice_rmu_ties %ld\n", ties);
  }
  return bad ? 1 : 0;
}

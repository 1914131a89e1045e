/*
 * oracle.c -- plain FP64 CPU reference for two-point pair counting.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; it is used by tests/, by __graft_entry__.smoke() and by
 * the cpu_baseline / --impl reference legs of bench.py.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (Alonso 2012, "CUTE solutions for two-point correlation
 * functions from large cosmological datasets"):
 *
 *   * the pair-count histogram of Sec. 2.2, Eq. 11: every pair of objects is
 *     examined, its separation computed, and the bin it falls in incremented;
 *     self-pairs are excluded.  Following the serial loop of Sec. 3.1, the
 *     count is a plain double loop over both catalogs.  Auto-correlations
 *     count each unordered pair {i,j}, i<j, once; cross-correlations count
 *     every (i in A, j in B).
 *   * the separation measures of Sec. 2.1: the monopole distance |x_j - x_i|,
 *     the (sigma, pi) split with pi along the line of sight (Eq. 2), the
 *     (r, mu) split with mu the cosine between the separation and the line of
 *     sight, and the angle between unit vectors (Eq. 7), measured here by the
 *     chord length |n_j - n_i| = 2 sin(theta/2), a monotone function of theta.
 *   * periodic boxes wrap each separation component to its minimum image
 *     (Sec. 2.2, the estimator of Eq. 13, and Sec. 3.4.4).
 *   * weighted counts sum w_i w_j over the pairs of each bin (the pixel and
 *     density-grid weights of Sec. 3.4), and the gradient of a weighted-count
 *     functional with respect to one object's weight.
 *   * the estimators: Eq. 13 (periodic box), Eq. 14 (natural), Eq. 15
 *     (Landy-Szalay).
 *
 * Readings where the paper is silent (the same readings are listed with the
 * design notes of the repository):
 *   - bins are half-open [e_b, e_{b+1}); comparisons are made on squared
 *     quantities, d^2 against e_b^2 (Eq. 11 writes open bounds on both sides);
 *   - out-of-range pairs are counted in a separate counter (the serial loop of
 *     Sec. 3.1 does not say what bin_dist returns for them);
 *   - histograms are 64-bit (the listings use int);
 *   - the line of sight is the pair midpoint x_i + x_j for (r, mu) on open
 *     (light-cone) catalogs and the z axis for (sigma, pi); mu is |cos| in
 *     [0,1] with the top edge mu = 1 inclusive; coincident points take mu bin 0;
 *   - Eq. 13 uses N(N-1)/2 unique pairs and the exact shell volume
 *     4pi/3 (r2^3 - r1^3), instead of N^2 and 4 pi r^2 dr.
 *
 * Canonical FP64 formulas (no FMA contraction: build with -ffp-contract=off):
 *   delta_k = x_j,k - x_i,k, wrapped once by +-L when |delta_k| > L/2 (periodic)
 *   d2      = (dx*dx + dy*dy) + dz*dz                    (monopole, chord^2)
 *   sigma2  = dx*dx + dy*dy,  pi2 = dz*dz                (sigma, pi)
 *   s = x_j - x_i, l = x_i + x_j, r2 = (s.s), L2 = (l.l), sl = (s.l) left to
 *   right, q = sl*sl, den = r2*L2; mu bin = largest k in [0, n_mu-1] with
 *   q >= (m_k*m_k)*den                                   (r, mu)
 *   bin b  <=>  e_b*e_b <= v < e_{b+1}*e_{b+1}
 *
 * Weighted sums are accumulated with Neumaier-compensated FP64 so the
 * oracle's own rounding stays far below the 1e-9 tolerance of the tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { K_MONO = 0, K_RMU = 1, K_SIGPI = 2, K_THETA = 3 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2 };

/* ---------------- compensated summation (Neumaier) ---------------- */
typedef struct { double s, c; } csum;

static void cs_add(csum *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double cs_val(const csum *a) { return a->s + a->c; }

/* ---------------- binning specification ---------------- */
typedef struct {
  int kind, periodic;
  double L, halfL;
  int n0, n1;          /* n1 = 1 for the 1-D kinds */
  double *E0, *E1;     /* squared edges, n0+1 and n1+1 values */
} spec;

static int spec_init(spec *s, int kind, int periodic, double L,
                     const double *e0, int n0, const double *e1, int n1) {
  if (kind < 0 || kind > 3 || n0 < 1 || !e0) return ORC_EINVAL;
  int two_d = (kind == K_RMU || kind == K_SIGPI);
  if (two_d && (n1 < 1 || !e1)) return ORC_EINVAL;
  if (periodic && !(L > 0)) return ORC_EINVAL;
  s->kind = kind; s->periodic = periodic; s->L = L; s->halfL = 0.5 * L;
  s->n0 = n0; s->n1 = two_d ? n1 : 1;
  s->E0 = (double *)malloc(sizeof(double) * (size_t)(n0 + 1));
  s->E1 = (double *)malloc(sizeof(double) * (size_t)(s->n1 + 1));
  if (!s->E0 || !s->E1) { free(s->E0); free(s->E1); return ORC_ENOMEM; }
  for (int k = 0; k <= n0; k++) {
    if (!(e0[k] >= 0) || (k > 0 && !(e0[k] > e0[k - 1]))) goto bad;
    s->E0[k] = e0[k] * e0[k];
  }
  if (two_d) {
    for (int k = 0; k <= n1; k++) {
      if (!(e1[k] >= 0) || (k > 0 && !(e1[k] > e1[k - 1]))) goto bad;
      s->E1[k] = e1[k] * e1[k];
    }
    /* mu covers [0,1] exactly */
    if (kind == K_RMU && (e1[0] != 0.0 || e1[n1] != 1.0)) goto bad;
  } else {
    s->E1[0] = 0; s->E1[1] = 0;
  }
  return ORC_OK;
bad:
  free(s->E0); free(s->E1);
  return ORC_EINVAL;
}
static void spec_free(spec *s) { free(s->E0); free(s->E1); }

/* bin b with E[b] <= v < E[b+1], or -1 when v is outside [E[0], E[n]) */
static int bin_of(const double *E, int n, double v) {
  if (!(v >= E[0]) || !(v < E[n])) return -1;
  int lo = 0, hi = n; /* E[lo] <= v < E[hi] */
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (v >= E[mid]) lo = mid; else hi = mid;
  }
  return lo;
}

/* largest k in [0, n-1] with q >= M[k]*den; M[0] = 0 so k = 0 always holds */
static int mu_bin_of(const double *M, int n, double q, double den) {
  int lo = 0, hi = n; /* q >= M[lo]*den holds; k >= hi fails */
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    double t = M[mid] * den;
    if (q >= t) lo = mid; else hi = mid;
  }
  return lo;
}

static double wrap(double d, const spec *s) {
  if (s->periodic) {
    if (d > s->halfL) d -= s->L;
    else if (d < -s->halfL) d += s->L;
  }
  return d;
}

/* flat bin index of the pair (a, b), or -1 when out of range */
static int pair_bin(const spec *s, const double *a, const double *b) {
  switch (s->kind) {
  case K_MONO:
  case K_THETA: {
    double dx = wrap(b[0] - a[0], s), dy = wrap(b[1] - a[1], s),
           dz = wrap(b[2] - a[2], s);
    double d2 = (dx * dx + dy * dy) + dz * dz;
    return bin_of(s->E0, s->n0, d2);
  }
  case K_SIGPI: {
    double dx = wrap(b[0] - a[0], s), dy = wrap(b[1] - a[1], s),
           dz = wrap(b[2] - a[2], s);
    double sg2 = dx * dx + dy * dy;
    double pi2 = dz * dz;
    int bs = bin_of(s->E0, s->n0, sg2);
    if (bs < 0) return -1;
    int bp = bin_of(s->E1, s->n1, pi2);
    if (bp < 0) return -1;
    return bs * s->n1 + bp;
  }
  case K_RMU: {
    double sx = b[0] - a[0], sy = b[1] - a[1], sz = b[2] - a[2];
    double lx = a[0] + b[0], ly = a[1] + b[1], lz = a[2] + b[2];
    double r2 = (sx * sx + sy * sy) + sz * sz;
    int br = bin_of(s->E0, s->n0, r2);
    if (br < 0) return -1;
    int bm;
    if (r2 == 0.0) {
      bm = 0;
    } else {
      double L2 = (lx * lx + ly * ly) + lz * lz;
      double sl = (sx * lx + sy * ly) + sz * lz;
      double q = sl * sl;
      double den = r2 * L2;
      bm = mu_bin_of(s->E1, s->n1, q, den);
    }
    return br * s->n1 + bm;
  }
  }
  return -1;
}

static int nthreads_of(int req) {
#ifdef _OPENMP
  return req > 0 ? req : omp_get_max_threads();
#else
  (void)req;
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Brute-force count: every pair examined (Sec. 3.1 serial loop, Eq. 11).
 * xa, xb: row-major n x 3 FP64.  is_auto: count i<j within xa (xb ignored).
 * counts: n0*n1 uint64 (row-major [axis0][axis1]); oor: pairs out of range;
 * wsum (optional, needs wa and wb, or wa alone for auto): sum of w_i w_j per
 * bin.  The outer loop is split across threads, each with a private
 * histogram, merged in thread order (Sec. 3.2.1). */
int oracle_count(int kind, int periodic, double L,
                 const double *xa, int64_t na, const double *xb, int64_t nb,
                 int is_auto, const double *e0, int n0, const double *e1,
                 int n1, const float *wa, const float *wb, uint64_t *counts,
                 uint64_t *oor, double *wsum, int nthreads) {
  spec s;
  int rc = spec_init(&s, kind, periodic, L, e0, n0, e1, n1);
  if (rc) return rc;
  if (na < 0 || nb < 0 || !counts || (na > 0 && !xa)) { spec_free(&s); return ORC_EINVAL; }
  if (is_auto) { xb = xa; nb = na; wb = wa; }
  else if (nb > 0 && !xb) { spec_free(&s); return ORC_EINVAL; }
  int want_w = (wsum != NULL);
  if (want_w && (!wa || !wb)) { spec_free(&s); return ORC_EINVAL; }
  const int nbins = s.n0 * s.n1;
  const int nt = nthreads_of(nthreads);
  uint64_t *hc = (uint64_t *)calloc((size_t)nt * (nbins + 1), sizeof(uint64_t));
  csum *hw = (csum *)calloc(want_w ? (size_t)nt * nbins : 1, sizeof(csum));
  if (!hc || !hw) { free(hc); free(hw); spec_free(&s); return ORC_ENOMEM; }

#pragma omp parallel num_threads(nt)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    uint64_t *mc = hc + (size_t)t * (nbins + 1);
    csum *mw = hw + (want_w ? (size_t)t * nbins : 0);
#pragma omp for schedule(static, 16)
    for (int64_t i = 0; i < na; i++) {
      const double *a = xa + 3 * i;
      int64_t j0 = is_auto ? i + 1 : 0;
      for (int64_t j = j0; j < nb; j++) {
        int b = pair_bin(&s, a, xb + 3 * j);
        if (b < 0) { mc[nbins]++; continue; }
        mc[b]++;
        if (want_w) cs_add(&mw[b], (double)wa[i] * (double)wb[j]);
      }
    }
  }
  uint64_t o = 0;
  for (int b = 0; b < nbins; b++) counts[b] = 0;
  for (int t = 0; t < nt; t++) {
    for (int b = 0; b < nbins; b++) counts[b] += hc[(size_t)t * (nbins + 1) + b];
    o += hc[(size_t)t * (nbins + 1) + nbins];
  }
  if (oor) *oor = o;
  if (want_w) {
    for (int b = 0; b < nbins; b++) {
      csum acc = {0, 0};
      for (int t = 0; t < nt; t++) {
        cs_add(&acc, hw[(size_t)t * nbins + b].s);
        cs_add(&acc, hw[(size_t)t * nbins + b].c);
      }
      wsum[b] = cs_val(&acc);
    }
  }
  free(hc); free(hw); spec_free(&s);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Cell-pruned count (Sec. 3.3): the volume is covered by cells no smaller
 * than the reach on each axis, and only pairs of cells that touch (or the
 * same cell) are examined; every other pair has some |delta_k| >= reach_k
 * and is out of range.  Each examined pair is binned with the same canonical
 * formula as the brute force, so the counts are identical.  reach[3]: the
 * largest separation per axis that can fall in a bin. */
typedef struct {
  int n[3];
  double lo[3], a[3];
  int64_t *start; /* ncell + 1 */
  int64_t *idx;   /* point indices grouped by cell */
} cellgrid;

static int cell_coord(double x, double lo, double a, int n) {
  double f = floor((x - lo) / a);
  int c = (f < 0) ? 0 : (f >= n ? n - 1 : (int)f);
  return c;
}

static int grid_build(cellgrid *g, const double *x, int64_t n) {
  int64_t nc = (int64_t)g->n[0] * g->n[1] * g->n[2];
  g->start = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
  g->idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t *cid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!g->start || !g->idx || !cid) { free(g->start); free(g->idx); free(cid); return ORC_ENOMEM; }
  for (int64_t i = 0; i < n; i++) {
    int cx = cell_coord(x[3 * i], g->lo[0], g->a[0], g->n[0]);
    int cy = cell_coord(x[3 * i + 1], g->lo[1], g->a[1], g->n[1]);
    int cz = cell_coord(x[3 * i + 2], g->lo[2], g->a[2], g->n[2]);
    cid[i] = ((int64_t)cz * g->n[1] + cy) * g->n[0] + cx;
    g->start[cid[i] + 1]++;
  }
  for (int64_t c = 0; c < nc; c++) g->start[c + 1] += g->start[c];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
  if (!fill) { free(g->start); free(g->idx); free(cid); return ORC_ENOMEM; }
  memcpy(fill, g->start, sizeof(int64_t) * (size_t)nc);
  for (int64_t i = 0; i < n; i++) g->idx[fill[cid[i]]++] = i;
  free(fill); free(cid);
  return ORC_OK;
}

/* distinct neighbour coordinates of cell c along one axis (at most 3) */
static int axis_neigh(int c, int n, int periodic, int out[3]) {
  int m = 0;
  for (int d = -1; d <= 1; d++) {
    int v = c + d;
    if (periodic) v = ((v % n) + n) % n;
    else if (v < 0 || v >= n) continue;
    int dup = 0;
    for (int k = 0; k < m; k++) dup |= (out[k] == v);
    if (!dup) out[m++] = v;
  }
  return m;
}

int oracle_count_cells(int kind, int periodic, double L,
                       const double *xa, int64_t na, const double *xb,
                       int64_t nb, int is_auto, const double *e0, int n0,
                       const double *e1, int n1, const float *wa,
                       const float *wb, const double *reach, uint64_t *counts,
                       uint64_t *oor, double *wsum, int nthreads) {
  spec s;
  int rc = spec_init(&s, kind, periodic, L, e0, n0, e1, n1);
  if (rc) return rc;
  if (na < 0 || nb < 0 || !counts || !reach || (na > 0 && !xa)) { spec_free(&s); return ORC_EINVAL; }
  if (is_auto) { xb = xa; nb = na; wb = wa; }
  else if (nb > 0 && !xb) { spec_free(&s); return ORC_EINVAL; }
  int want_w = (wsum != NULL);
  if (want_w && (!wa || !wb)) { spec_free(&s); return ORC_EINVAL; }

  /* geometry shared by both catalogs */
  cellgrid ga, gb;
  memset(&ga, 0, sizeof ga); memset(&gb, 0, sizeof gb);
  for (int k = 0; k < 3; k++) {
    double lo, hi;
    if (periodic) { lo = 0; hi = L; }
    else {
      lo = INFINITY; hi = -INFINITY;
      for (int64_t i = 0; i < na; i++) { lo = fmin(lo, xa[3 * i + k]); hi = fmax(hi, xa[3 * i + k]); }
      for (int64_t j = 0; j < nb; j++) { lo = fmin(lo, xb[3 * j + k]); hi = fmax(hi, xb[3 * j + k]); }
      if (!(hi >= lo)) { lo = 0; hi = 1; }
    }
    double ext = hi - lo;
    /* cells at least reach*(1+1e-9) wide, so two points whose cells are two
       or more apart differ by at least the reach on that axis */
    double amin = reach[k] * (1.0 + 1e-9) + 1e-300;
    int n = (int)floor(ext / amin);
    if (n < 1) n = 1;
    if (periodic && n < 3) n = 1; /* too few cells to prune on this axis */
    if (n > 128) n = 128; /* coarser cells still prune correctly */
    ga.n[k] = gb.n[k] = n;
    ga.lo[k] = gb.lo[k] = lo;
    ga.a[k] = gb.a[k] = (periodic ? ext / n : fmax(ext / n, amin));
  }
  if (grid_build(&ga, xa, na) || grid_build(&gb, xb, nb)) {
    free(ga.start); free(ga.idx); free(gb.start); free(gb.idx); spec_free(&s);
    return ORC_ENOMEM;
  }
  const int nbins = s.n0 * s.n1;
  const int nt = nthreads_of(nthreads);
  const int64_t ncell = (int64_t)ga.n[0] * ga.n[1] * ga.n[2];
  uint64_t *hc = (uint64_t *)calloc((size_t)nt * (nbins + 1), sizeof(uint64_t));
  csum *hw = (csum *)calloc(want_w ? (size_t)nt * nbins : 1, sizeof(csum));
  if (!hc || !hw) {
    free(hc); free(hw); free(ga.start); free(ga.idx); free(gb.start); free(gb.idx);
    spec_free(&s); return ORC_ENOMEM;
  }
#pragma omp parallel num_threads(nt)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    uint64_t *mc = hc + (size_t)t * (nbins + 1);
    csum *mw = hw + (want_w ? (size_t)t * nbins : 0);
#pragma omp for schedule(dynamic, 1)
    for (int64_t c1 = 0; c1 < ncell; c1++) {
      int cx = (int)(c1 % ga.n[0]), cy = (int)((c1 / ga.n[0]) % ga.n[1]),
          cz = (int)(c1 / ((int64_t)ga.n[0] * ga.n[1]));
      int nx[3], ny[3], nz[3];
      int mx = axis_neigh(cx, ga.n[0], periodic, nx);
      int my = axis_neigh(cy, ga.n[1], periodic, ny);
      int mz = axis_neigh(cz, ga.n[2], periodic, nz);
      for (int iz = 0; iz < mz; iz++)
        for (int iy = 0; iy < my; iy++)
          for (int ix = 0; ix < mx; ix++) {
            int64_t c2 = ((int64_t)nz[iz] * ga.n[1] + ny[iy]) * ga.n[0] + nx[ix];
            if (is_auto && c2 < c1) continue;
            for (int64_t p = ga.start[c1]; p < ga.start[c1 + 1]; p++) {
              int64_t i = ga.idx[p];
              const double *a = xa + 3 * i;
              int64_t q0 = gb.start[c2];
              if (is_auto && c2 == c1) q0 = p + 1;
              for (int64_t q = q0; q < gb.start[c2 + 1]; q++) {
                int64_t j = gb.idx[q];
                int b = pair_bin(&s, a, xb + 3 * j);
                if (b < 0) continue;
                mc[b]++;
                if (want_w) cs_add(&mw[b], (double)wa[i] * (double)wb[j]);
              }
            }
          }
    }
  }
  uint64_t inrange = 0;
  for (int b = 0; b < nbins; b++) counts[b] = 0;
  for (int t = 0; t < nt; t++)
    for (int b = 0; b < nbins; b++) counts[b] += hc[(size_t)t * (nbins + 1) + b];
  for (int b = 0; b < nbins; b++) inrange += counts[b];
  uint64_t total = is_auto ? (uint64_t)na * (uint64_t)(na > 0 ? na - 1 : 0) / 2
                           : (uint64_t)na * (uint64_t)nb;
  if (oor) *oor = total - inrange;
  if (want_w) {
    for (int b = 0; b < nbins; b++) {
      csum acc = {0, 0};
      for (int t = 0; t < nt; t++) {
        cs_add(&acc, hw[(size_t)t * nbins + b].s);
        cs_add(&acc, hw[(size_t)t * nbins + b].c);
      }
      wsum[b] = cs_val(&acc);
    }
  }
  free(hc); free(hw); free(ga.start); free(ga.idx); free(gb.start); free(gb.idx);
  spec_free(&s);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Gradient rows of the weighted-count functional
 *   F(w) = sum_b G_b W_b,   W_b = sum over pairs in bin b of w_i w_j,
 * with respect to the weight of object i of catalog A:
 *   dF/dw_i = sum_{j != i} w_j G[bin(i,j)]   (auto, partners in A)
 *   dF/dw_i = sum_j w^B_j G[bin(i,j)]        (cross, partners in B).
 * For the gradient with respect to catalog B's weights of a cross count,
 * call with the catalogs swapped (the canonical bin is symmetric).
 * rows: indices into A; grad: one FP64 value per row. */
int oracle_grad_rows(int kind, int periodic, double L, const double *xa,
                     int64_t na, const double *xb, int64_t nb, int is_auto,
                     const double *e0, int n0, const double *e1, int n1,
                     const float *wpartner, const double *G,
                     const int64_t *rows, int64_t nrows, double *grad,
                     int nthreads) {
  spec s;
  int rc = spec_init(&s, kind, periodic, L, e0, n0, e1, n1);
  if (rc) return rc;
  if (is_auto) { xb = xa; nb = na; }
  if (!G || !wpartner || !grad || (nrows > 0 && !rows) || !xa || (nb > 0 && !xb)) {
    spec_free(&s); return ORC_EINVAL;
  }
  for (int64_t r = 0; r < nrows; r++)
    if (rows[r] < 0 || rows[r] >= na) { spec_free(&s); return ORC_EINVAL; }
  const int nt = nthreads_of(nthreads);
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; r++) {
    int64_t i = rows[r];
    const double *a = xa + 3 * i;
    csum acc = {0, 0};
    for (int64_t j = 0; j < nb; j++) {
      if (is_auto && j == i) continue;
      /* auto pairs are binned in index order (lower index first), as counted */
      int b = (is_auto && j < i) ? pair_bin(&s, xb + 3 * j, a)
                                 : pair_bin(&s, a, xb + 3 * j);
      if (b < 0) continue;
      cs_add(&acc, (double)wpartner[j] * G[b]);
    }
    grad[r] = cs_val(&acc);
  }
  spec_free(&s);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Estimators (Sec. 2.2).  Counts are unique pairs; bins with a zero
 * denominator give NaN.
 *   periodic (Eq. 13, exact shell):  xi_b = DD_b / (N(N-1)/2 * V_b / L^3) - 1,
 *                                    V_b = 4pi/3 (e_{b+1}^3 - e_b^3)
 *   natural  (Eq. 14):  xi = Nr(Nr-1)/(Nd(Nd-1)) DD/RR - 1
 *   Landy-Szalay (Eq. 15):
 *     xi = (Nr(Nr-1)/(Nd(Nd-1)) DD - (Nr-1)/Nd DR + RR) / RR            */
int oracle_xi_periodic(const uint64_t *DD, int64_t N, const double *edges,
                       int nbins, double L, double *xi) {
  if (!DD || !edges || !xi || nbins < 1 || !(L > 0) || N < 2) return ORC_EINVAL;
  const double pi = 3.14159265358979323846;
  double npairs = 0.5 * (double)N * (double)(N - 1);
  double vol = L * L * L;
  for (int b = 0; b < nbins; b++) {
    double r1 = edges[b], r2 = edges[b + 1];
    double shell = (4.0 * pi / 3.0) * (r2 * r2 * r2 - r1 * r1 * r1);
    double expect = npairs * shell / vol;
    xi[b] = (expect > 0) ? (double)DD[b] / expect - 1.0 : NAN;
  }
  return ORC_OK;
}

int oracle_xi_natural(const uint64_t *DD, const uint64_t *RR, int64_t Nd,
                      int64_t Nr, int nbins, double *xi) {
  if (!DD || !RR || !xi || nbins < 1 || Nd < 2 || Nr < 2) return ORC_EINVAL;
  double f = ((double)Nr * (double)(Nr - 1)) / ((double)Nd * (double)(Nd - 1));
  for (int b = 0; b < nbins; b++)
    xi[b] = RR[b] ? f * (double)DD[b] / (double)RR[b] - 1.0 : NAN;
  return ORC_OK;
}

int oracle_xi_ls(const uint64_t *DD, const uint64_t *DR, const uint64_t *RR,
                 int64_t Nd, int64_t Nr, int nbins, double *xi) {
  if (!DD || !DR || !RR || !xi || nbins < 1 || Nd < 2 || Nr < 2) return ORC_EINVAL;
  double f = ((double)Nr * (double)(Nr - 1)) / ((double)Nd * (double)(Nd - 1));
  double g = (double)(Nr - 1) / (double)Nd;
  for (int b = 0; b < nbins; b++) {
    if (!RR[b]) { xi[b] = NAN; continue; }
    xi[b] = (f * (double)DD[b] - g * (double)DR[b] + (double)RR[b]) / (double)RR[b];
  }
  return ORC_OK;
}

/* chord length between two unit vectors separated by theta (degrees):
   |n_1 - n_2| = 2 sin(theta/2)  (Eq. 7 gives cos theta = n_1 . n_2) */
int oracle_theta_to_chord(const double *theta_deg, int n, double *chord) {
  if (!theta_deg || !chord || n < 0) return ORC_EINVAL;
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; k++) chord[k] = 2.0 * sin(0.5 * theta_deg[k] * (pi / 180.0));
  return ORC_OK;
}

int oracle_max_threads(void) { return nthreads_of(0); }

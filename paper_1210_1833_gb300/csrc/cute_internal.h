// cute_internal.h -- structures shared by the host planner and the kernels
// of libcute_gb.so.  Not part of the public ABI (see include/cute.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>
#include <map>
#include <memory>

#include <cuda_runtime.h>

#include "../../include/cute.h"

namespace cute {

// ------------------------------------------------------------------ binning
// Each binning axis maps an FP32 value v (a squared separation, or mu) to a
// cell of a lookup table.  Every axis has slots 0..nb+1: slot 0 below the
// first edge, slot b+1 for bin b, slot nb+1 above the last edge (0 and nb+1
// collect out-of-range pairs and are never reported).  A table entry holds
// the byte offset of a histogram slot (bits 0..19) and a band index (bits
// 20..31).  Band 0: the cell is CLEAN -- every value in it, widened by the
// proven FP32 error bound, lies strictly between the same two edges, so the
// offset is the pair's slot.  Band k+1: the cell meets the error band of edge
// k only; the offset is the slot just below edge k, values above the band
// take the next slot, values inside it are re-tested (double-float, then FP64).  The last band
// index of an axis marks cells that always go to FP64.
constexpr uint32_t kOffMask = 0xFFFFu;     // slot byte offset (bits 0..15)
constexpr int kClassShift = 16;            // R_MU r entries: mu error class (bits 16..19)
constexpr int kBandShift = 20;             // band index (bits 20..31)
constexpr int kLutLinear = 0;              // idx = rne(v * scale)
constexpr int kLutLog = 1;                 // idx = max((bits(v) >> shift) - base, 0)
constexpr int kArith = 2;                  // uniform edges: bin = floor((x - e0) / delta)
constexpr int kArithLog = 3;               // log-spaced edges: t from log2(v) (monopole, chords)
constexpr int kArithLogU = 4;              // the same without the upper clamp: spare slots above
                                           // the last bin hold every t a pair can reach

struct AxisPlan {
  int mode = 0;
  int ncell = 0;      // table cells
  float vmax = 0;     // values are clamped to [.., vmax] before lookup
  float scale = 0;    // linear mode
  int shift = 0;      // log mode
  int base = 0;       // log mode
  int lut_off = 0;    // word offset of this axis in the table block
  int nb = 0;         // bins on the axis
  int band_off = 0;   // float2 offset of this axis's bands in the band table
  int nband = 0;      // bands of this axis (nb + 3: none, one per edge, always)
  // kArith: t = x * inv + cst (cst already holds -e0/delta - 1/2), clamped
  // above to thi (tlo is the planner's bookkeeping only);
  // the bin is rint(t) and the pair is near an edge when
  // |t - rint(t)| + thr >= 1/2, with thr = thr_a / x_r + thr_b for mu
  // (x_r the pair's r) and thr_b alone for the other axes.
  float inv = 0, cst = 0, tlo = 0, thi = 0, thr_a = 0, thr_b = 0;
  float near_at = 0;  // 1/2 - thr_b rounded down: near when |h| >= near_at
  // mu: 1/2 - thr_b - 2^-22 rounded down; near when |h| >= near_c - thr_a * rr
  // (one FMA, its rounding covered by the 2^-22)
  float near_c = 0;
  // (sigma, pi), axis 1: near_at(axis 0) / near_at(axis 1) rounded up
  float near_scale = 1;
  // kArithLog: t = inv log2(max(v, vlo)) + (ld v + lb) v + cst, clamped
  // above to thi; near when |h| + thr_a / sqrt(v) reaches near_c (as mu)
  float lb = 0, ld = 0, vlo = 0;
  // (r, mu), axis 1: scale k of the squared line-of-sight length the kernel
  // forms (k = 1/inv^2 rounded, so |s.l| / sqrt(r^2 k l^2) is mu * inv;
  // 1 for tables)
  float lsc = 1;
};

// Kinds as the kernels see them.
constexpr int KMONO = 0, KRMU = 1, KSIGPI = 2, KTHETA = 3;

// Work decomposition.  Catalog A is cut into home CHUNKS of at most
// 32 x home_per_lane objects that lie in one row of cells (cx0..cx1, cy, cz);
// the STENCIL lists the neighbour rows (dy, dz) a chunk can reach, each with
// the x-extent kxr.  A work ENTRY is (chunk, stencil row): the chunk against
// the objects of catalog B in that row, in at most three contiguous
// SEGMENTS (the home cell run itself with j > i on the home row of an auto
// count, and the row's x-range split where it wraps around a periodic box).
// A segment splits into slices of at most `slice` neighbours: one work item
// each, written as a 16-byte record (item_record) on the GPU.
//   chunk int4: (h0, h1, cx0 | cx1 << 16, cy | cz << 16)
//   stencil row int4: (dy, dz, kxr, 1 on the home row)
constexpr int kSegSelf = 1;        // only j > i (unique pairs of a run with itself)
constexpr int kSegNoSelfPair = 2;  // every j != i (full-stencil adjoint of an auto count)
constexpr int kCounterWords = 7;  // work ticket + 6 statistics words
constexpr int kMaxDevices = 64;   // per-device launch caches
// Warps per block (one block per SM) the counting kernel is compiled for:
// the plain monopole / chord count with two home objects per lane fits in
// 96 registers and may run 20 warps; every other instantiation 16.
constexpr int count_max_warps(int kernel_kind_mono, int hp, int acc) {
  return (kernel_kind_mono && hp == 2 && acc == 0) ? 20 : 16;
}
constexpr int kModeCross = 0, kModeAutoHalf = 1, kModeAutoFull = 2;

// One pair set (cat_a, cat_b) of a (possibly batched) count, as the
// counting kernel sees it.
// Double-float view of a pair set for the first stage of the re-test: the
// FP32 frame offsets plus their FP32 remainders (pos + lo = x - fo to
// about 2^-48 |x - fo|) and the absolute error bounds of the separation and
// line-of-sight components formed from them.
struct PairDF {
  const float4 *loA, *loB;     // cell-sorted remainders (x, y, z, 0)
  float eta;                   // bound on the error of a separation component
  float eta_l;                 // R_MU: of a line-of-sight component (x_i + x_j)
  float Lh, Ll;                // periodic box as hi + lo (0 when open)
  float fo2h[3], fo2l[3];      // R_MU: twice the frame centre (observer frame), hi + lo
};

struct PairDev {
  const float4 *posA, *posB;   // cell-sorted FP32 (x, y, z, w), grid frame
  // R_MU: cell-sorted FP32 (x, y, z, q), q = |x|^2 - q0 in the observer frame
  // (rounded once from FP64); null for periodic grids
  const float4 *qA, *qB;
  double q0;                   // R_MU: reference of q (the geometry's)
  const double *sA, *sB;       // cell-sorted FP64 SoA (x[n], y[n], z[n])
  const PairDF *df;            // double-float view (re-test first stage)
  const int32_t *permA;        // cell-sorted index -> upload index of A
  int32_t nA, nB;
  int32_t out;                 // output histogram index
  int32_t is_auto;
  float L32;                   // periodic box as FP32 (image shifts)
  double L64;                  // periodic box in FP64, 0 for open
};

// The same pair set as the work builder sees it.
struct PairWork {
  const int4 *chunks;          // home chunks of A
  const int4 *stencil;         // stencil rows
  const int32_t *csB;          // cell_start of B (ncell + 1)
  int32_t nchunks, nstencil;
  int32_t nx, ny, nz;          // cells per axis
  int32_t mode;                // kModeCross / kModeAutoHalf / kModeAutoFull
  int32_t periodic;
};

struct KParams {
  const int4 *items;           // work item records
  long long total;             // work items handed out
  long long item_stride;       // record of ticket t: items[t * item_stride] (1; the
                               // autotuner times an evenly spread sample)
  const PairDev *pairs;
  const uint32_t *lut;         // table words, all axes
  int lut_words;
  AxisPlan ax[2];
  const float2 *band;          // (lo, hi) per band, both axes, FP32, outward rounded;
                               // mu bands hold (edge, edge)
  int band_words;              // float2 entries in band
  float mu_eps_base;           // R_MU: mu error bound of class 0 (class c: x 2^c)
  // padded home slots sit at +far and padded tile rows at -far on every axis
  // of the FP32 grid frame: beyond any reach, every product finite
  float far;
  // integer weights (kAccIntWeighted): the largest weight product, for the
  // uint32 overflow guard of the per-bin weight sums
  unsigned wpmax;
  // neighbour cull: a tile row of another cell is skipped when its FP32
  // distance from the bounding box of the item's home objects exceeds the
  // reach -- squared, cull_r2 (sigma, pi: cull_r2 in x-y and cull_pi along
  // z) -- both widened past every rounding of the FP32 frame (cull_params)
  float cull_r2, cull_pi;
  const double *E0, *E1;       // FP64 squared edges (mu: squared mu edges)
  const float2 *E0df, *E1df;   // the same as FP32 hi + lo
  int n0, n1;                  // bins per axis (n1 = 1 for 1-D kinds)
  int slots1;                  // axis-1 slots (n1 + 2), 1 for 1-D kinds
  int nslots;                  // (n0 + 2) * slots1
  int R;                       // histogram copies per warp (power of 2, <= 32)
  int slice;                   // neighbour objects per work item
  unsigned long long *out_counts;  // [nout][n0 * n1]
  double *out_wsum;                // [nout][n0 * n1] or null
  unsigned long long *ticket;      // work-item counter
  unsigned long long *stats;       // [0] rechecked, [1] items, [2] near-band, [3] pair slots,
                                   // [4] candidate pairs, [5] decided by the FP64 formula
  // (ticket and stats are kCounterWords consecutive words, zeroed per launch)
  int *err;                        // first error code seen by a kernel
  // adjoint
  const double *G;                 // [n0 * n1] upstream gradient
  double *grad;                    // per sorted object of A
};

// ------------------------------------------------------------------ host objects
// x cells per y/z cell size (grid.cu): rows of cells run along x
constexpr int kXFine = 8;

struct Geometry {
  int id = 0;
  int periodic = 0;
  double L = 0;
  double origin[3] = {0, 0, 0};
  double a[3] = {1, 1, 1};
  int nc[3] = {1, 1, 1};
  int k[3] = {1, 1, 1};       // cells per reach on each axis
  int kreq = 2;               // cells per reach requested
  double reach[3] = {0, 0, 0};
  double xmax[3] = {0, 0, 0}; // largest |x - fo| per axis over its catalogs
  double fo[3] = {0, 0, 0};   // centre of the FP32 frame
  double absmax[3] = {0, 0, 0}; // largest |x| (observer frame) per axis
  double rmin = 0;            // smallest |x| over its catalogs (observer frame)
  double rmax = 0;            // largest |x| over its catalogs (observer frame)
  // R_MU: reference q0 of the squared distances q = |x|^2 - q0 (the middle
  // of [rmin^2, rmax^2]) and a bound qd >= |q| over its catalogs
  double q0 = 0, qd = 0;
  long long version = 0;
};

struct Catalog {
  int32_t id = 0;
  int64_t n = 0;
  int boundary = CUTE_OPEN;
  double L = 0;
  double *d_xyz = nullptr;     // upload order, row-major n x 3
  float *d_w = nullptr;        // upload order weights, or null
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, absmax[3] = {0, 0, 0};
  double rmin = 0, rmax = 0;   // smallest and largest |x| (observer frame)
  // weights that are all integers in [0, 2048] (counts per pixel or cell):
  // their largest value; -1 for other weights or none
  int wint = -1;
  // grid
  int geom = -1;
  long long grid_version = 0;
  float4 *d_pos = nullptr;     // sorted FP32
  float4 *d_posq = nullptr;    // sorted FP32 (x, y, z, |x|^2 - q0), open grids only
  float4 *d_lo = nullptr;      // sorted FP32 remainders of the frame offsets
  double *d_s64 = nullptr;     // sorted FP64 SoA
  int32_t *d_perm = nullptr;   // sorted -> upload index
  int32_t *d_cell_start = nullptr;
  int32_t *h_cell_start = nullptr;  // host copy (ncell + 1), pinned, the context's
  size_t h_cap = 0;                 // ints in that pinned block
  int64_t occupied_cells = 0;  // cells holding at least one object
  // home chunks of this grid per chunk size (built on first use)
  mutable std::map<int, std::vector<int4>> chunk_cache;
};

struct Plan;  // binning plan (plan.cpp)

// The work decomposition of a (possibly batched) count on the device:
// chunks, stencils and pair descriptors built on the host, entry item counts
// and their prefix sums computed on the GPU.  Cached per set of catalogs and
// launch shape.
struct WorkSet {
  cudaStream_t st = nullptr;       // the context's stream: device arrays are pool blocks
  std::vector<PairDev> pairs;
  std::vector<PairDF> pdf;
  std::vector<PairWork> work;
  std::vector<int> ebase;          // npairs + 1
  int nentries = 0;
  int4 *d_chunks = nullptr, *d_stencil = nullptr;
  PairDev *d_pairs = nullptr;
  PairDF *d_pdf = nullptr;
  PairWork *d_work = nullptr;
  int *d_ebase = nullptr;
  int *d_cnt = nullptr;            // items per entry
  long long *d_bsum = nullptr;     // scan block sums
  long long *d_eprefix = nullptr;  // nentries + 1
  long long items = 0;             // work items
  int4 *d_items = nullptr;         // their records
  // pairs the items present (candidate pairs before the kernel's neighbour
  // cull): host copy, and the device word the work builder sums into
  unsigned long long stencil_pairs = 0;
  unsigned long long *d_spairs = nullptr;
  ~WorkSet() {
    for (void *q : {(void *)d_chunks, (void *)d_stencil, (void *)d_pairs, (void *)d_pdf,
                    (void *)d_work, (void *)d_ebase, (void *)d_cnt, (void *)d_bsum,
                    (void *)d_eprefix, (void *)d_items, (void *)d_spairs})
      if (q) cudaFreeAsync(q, st);
  }
};

}  // namespace cute

struct cute_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // stream-ordered pool for catalogs, grids and work lists: freed blocks stay
  // cached for the next request (no synchronising cudaMalloc/cudaFree per
  // upload, grid or count)
  cudaMemPool_t pool = nullptr;
  // pinned host blocks for the grids' host copies of cell_start, kept for
  // reuse by size
  std::multimap<size_t, int32_t *> pinned_free;
  int sm_count = 0;
  size_t smem_optin = 0;
  std::string err;
  int next_cat = 1;
  int next_geom = 1;
  long long version_counter = 0;
  std::map<int32_t, cute::Catalog> cats;
  std::map<int, cute::Geometry> geoms;
  // scratch owned by the context
  unsigned long long *d_ticket = nullptr;   // [0] ticket, [1..] stats
  int *d_err = nullptr;
  void *d_scratch = nullptr;                // grows as needed
  size_t scratch_bytes = 0;
  // launch overrides
  int hp_override = 0, warps_override = 0, slice_override = 0;
  bool table_binning = false;
  bool timing = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cute_stats stats{};
  // caches
  std::map<std::string, std::shared_ptr<cute::Plan>> plans;
  std::map<std::string, std::shared_ptr<cute::WorkSet>> work_cache;
  // autotuned launch shapes per (kind, catalogs, policy)
  std::map<std::string, cute_tuning> tuned;
  // CUDA graphs of batched counts with device outputs, replayed when the
  // same request comes again; captured on a private stream
  cudaStream_t cap_stream = nullptr;
  std::map<std::string, cudaGraphExec_t> graphs;
  void clear_caches() {
    for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
    work_cache.clear();
  }
};

namespace cute {

// host planner (plan.cpp)
struct Plan {
  int kind = 0;
  int n0 = 0, n1 = 1;
  int slots1 = 1, nslots = 0;
  int R = 1;
  AxisPlan ax[2];
  std::vector<uint32_t> lut;        // all axes
  std::vector<float> band;          // (lo, hi) per band, both axes
  float mu_eps_base = 0;            // R_MU
  float far = 1.0e9f;               // padding sentinel magnitude (KParams::far)
  std::vector<double> E0, E1;       // FP64 squared edges
  double dirty_frac[2] = {0, 0};    // expected fraction of pairs in dirty cells
  // device copies
  uint32_t *d_lut = nullptr;
  float *d_band = nullptr;
  double *d_E0 = nullptr, *d_E1 = nullptr;
  std::vector<float> E0df, E1df;    // (hi, lo) per edge
  float *d_E0df = nullptr, *d_E1df = nullptr;
  ~Plan();
};

struct ErrorParams {
  double eta0;      // per-component absolute FP32 error bound, without the |delta| term
  double lmin;      // R_MU: lower bound of |l| for pairs within reach
  double qd;        // R_MU: bound on |q| = ||x|^2 - q0| over the catalogs
  double q0;        // R_MU: largest reference q0 of the pair sets
  double xm;        // largest |x - frame centre| per axis over the pair sets (FP32 frame)
};

// Build the binning plan.  hist_budget_bytes: per-warp histogram budget.
std::string plan_build(int kind, const double *e0, int n0, const double *e1, int n1,
                       const ErrorParams &ep, int lut_budget_words, size_t hist_budget_bytes,
                       bool allow_arith, Plan &out);

// A validated pair descriptor (api.cu).
struct DescInfo {
  int kind;        // KMONO / KRMU / KSIGPI / KTHETA
  Catalog *A, *B;
  const Geometry *g;
  bool is_auto;
  double need[3];
};
cute_status validate_desc(cute_ctx *ctx, const cute_pair_desc *d, DescInfo &di);
double row_density(const Catalog &A, const Geometry &g);
ErrorParams error_params(const std::vector<DescInfo> &dis, double rmax);
double decision_reach(const cute_pair_desc *d);
// device blocks from the context's pool, ordered on its stream
cudaError_t dev_alloc(cute_ctx *ctx, void **p, size_t bytes);
void dev_free(cute_ctx *ctx, void *p);
// pinned host ints from the context's free blocks (at least n), and back
cudaError_t pinned_get(cute_ctx *ctx, size_t n, int32_t **p, size_t *cap);
void pinned_put(cute_ctx *ctx, int32_t *p, size_t cap);
PairDF pair_df(const DescInfo &di);
// The kernel's view of pair set `out` (catalogs, sizes, box, (r, mu) data).
PairDev pair_dev(const DescInfo &di, int out);
// The neighbour cull's radii for the pair sets of one launch (KParams).
void cull_params(const std::vector<DescInfo> &dis, const cute_pair_desc *d, int n, KParams &p);

// Home chunks of catalog A (plan.cpp): each row of cells cut into chunks of
// home_chunk objects (the last one of a row shorter), spanning at most
// `maxrun` cells (chunks_maxrun).
int chunks_maxrun(const Geometry &g);
void chunks_build(const Geometry &g, const int32_t *csA, int home_chunk,
                  std::vector<int4> &out);
// Neighbour stencil (plan.cpp).  shape: the region of separations that can
// fall in a bin, used to trim neighbour rows.  Auto counts without
// full_stencil keep the home row and the rows after it.
constexpr int kShapeBox = 0, kShapeBall = 1, kShapeDiskSlab = 2;
void stencil_build(const Geometry &g, bool is_auto, bool full_stencil, int shape,
                   const double need[3], std::vector<int4> &out);

// Work entries on the GPU (work.cu): work_count computes the item count of
// every entry and their exclusive prefix sums into eprefix[0..nentries]
// (bsum needs work_bsum_words(nentries) words); work_write then writes the
// item records of every entry at its prefix.  work_count also sums into
// *spairs the pairs the entries present to the counting kernel.
int work_bsum_words(int nentries);
cudaError_t work_count(const PairWork *d_pairs, const int *d_ebase, int npairs, int nentries,
                       int slice, int *d_cnt, long long *d_bsum, long long *d_eprefix,
                       unsigned long long *d_spairs, cudaStream_t st);
cudaError_t work_write(const PairWork *d_pairs, const int *d_ebase, int npairs, int nentries,
                       int slice, const long long *d_eprefix, int4 *d_items, cudaStream_t st);

}  // namespace cute

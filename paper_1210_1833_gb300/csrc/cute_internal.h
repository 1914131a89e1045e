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
// cell of a lookup table; the table entry is either the byte offset of the
// histogram slot the pair belongs to ("clean" cell: every value in the cell,
// widened by the proven FP32 error bound, lies strictly between the same two
// edges) or a DIRTY marker naming the one edge whose error band meets the
// cell.  Slot 0 of each axis collects out-of-range pairs; bin b is slot b+1.
constexpr uint32_t kDirty = 0x40000000u;   // entry >= kDirty: refine
constexpr uint32_t kAlways = 0x1u;         // with kDirty: always FP64 re-test
constexpr int kLutLinear = 0;              // idx = rne(v * scale)
constexpr int kLutLog = 1;                 // idx = max((bits(v) >> shift) - base, 0)

struct AxisPlan {
  int mode = 0;
  int ncell = 0;      // table cells
  float vmax = 0;     // values are clamped to [.., vmax] before lookup
  float scale = 0;    // linear mode
  int shift = 0;      // log mode
  int base = 0;       // log mode
  int lut_off = 0;    // word offset of this axis in the table block
  int nb = 0;         // bins on the axis
  int band_off = 0;   // offset (floats) of this axis's (lo, hi) band pairs
  int decision_lo = 0;  // first edge index that is a decision boundary
};

// Kinds as the kernels see them.
constexpr int KMONO = 0, KRMU = 1, KSIGPI = 2, KTHETA = 3;

// A task: the home objects [h0,h1) of catalog A (a run of cells of one row)
// against one contiguous slice [j0,j1) of catalog B (one row of neighbour
// cells), with one periodic image shift.  The kernel splits it into
// n_hc x n_sc work items of at most (32 x home_per_lane) x slice pairs.
struct Task {
  int32_t h0, h1, j0, j1;
  int32_t pair;    // index of the PairDev this task belongs to
  int32_t flags;   // bit 0: self (only j > i); bits 8..13: image shift code
  int32_t n_hc, n_sc;
};
constexpr int kTaskSelf = 1;

// One pair set (cat_a, cat_b) of a (possibly batched) count.
struct PairDev {
  const float4 *posA, *posB;   // cell-sorted FP32 (x, y, z, w), grid frame
  const double *sA, *sB;       // cell-sorted FP64 SoA (x[n], y[n], z[n])
  int32_t nA, nB;
  int32_t out;                 // output histogram index
  int32_t is_auto;
  float L32;                   // periodic box as FP32 (image shifts)
  double L64;                  // periodic box in FP64, 0 for open
};

struct KParams {
  const Task *tasks;
  const long long *prefix;     // ntasks + 1 work-item prefix sums
  int ntasks;
  long long total;             // work items
  const PairDev *pairs;
  const uint32_t *lut;         // table words, all axes
  int lut_words;
  AxisPlan ax[2];
  const float *band;           // (lo, hi) per edge per axis, FP32, outward rounded
  const float *mu_eps;         // per r slot: FP32 error bound of mu (R_MU)
  const float *mu_edge;        // FP32 mu edges (R_MU)
  const double *E0, *E1;       // FP64 squared edges (mu: squared mu edges)
  int n0, n1;                  // bins per axis (n1 = 1 for 1-D kinds)
  int slots1;                  // axis-1 slots (n1 + 1), 1 for 1-D kinds
  int nslots;                  // (n0 + 1) * slots1
  int R;                       // histogram copies per warp (power of 2, <= 32)
  int slice;                   // neighbour objects per work item
  float eps_main;              // R_MU: mu error bound the mu table was built for
  unsigned long long *out_counts;  // [nout][n0 * n1]
  double *out_wsum;                // [nout][n0 * n1] or null
  unsigned long long *ticket;      // work-item counter
  unsigned long long *stats;       // [0] rechecked pairs, [1] items run
  int *err;                        // first error code seen by a kernel
  // adjoint
  const double *G;                 // [n0 * n1] upstream gradient
  double *grad;                    // per sorted object of A
};

// ------------------------------------------------------------------ host objects
struct Geometry {
  int id = 0;
  int periodic = 0;
  double L = 0;
  double origin[3] = {0, 0, 0};
  double a[3] = {1, 1, 1};
  int nc[3] = {1, 1, 1};
  int k[3] = {1, 1, 1};       // cells per reach on each axis
  double reach[3] = {0, 0, 0};
  double xmax[3] = {0, 0, 0}; // largest |x - origin| per axis over its catalogs
  double absmax[3] = {0, 0, 0}; // largest |x| (observer frame) per axis
  double rmin = 0;            // smallest |x| over its catalogs (observer frame)
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
  double rmin = 0;
  // grid
  int geom = -1;
  long long grid_version = 0;
  float4 *d_pos = nullptr;     // sorted FP32
  double *d_s64 = nullptr;     // sorted FP64 SoA
  int32_t *d_perm = nullptr;   // sorted -> upload index
  int32_t *d_cell_start = nullptr;
  std::vector<int32_t> h_cell_start;
};

struct Plan;  // binning plan (plan.cpp)

// Device copy of the tasks, work-item prefix sums and pair descriptors of a
// (possibly batched) count; cached per set of catalogs and launch shape.
struct TaskSet {
  std::vector<Task> tasks;
  std::vector<long long> prefix;
  std::vector<PairDev> pairs;
  unsigned long long candidates = 0;
  Task *d_tasks = nullptr;
  long long *d_prefix = nullptr;
  PairDev *d_pairs = nullptr;
  ~TaskSet() {
    cudaFree(d_tasks);
    cudaFree(d_prefix);
    cudaFree(d_pairs);
  }
};

}  // namespace cute

struct cute_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
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
  bool timing = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cute_stats stats{};
  // caches
  std::map<std::string, std::shared_ptr<cute::Plan>> plans;
  std::map<std::string, std::shared_ptr<cute::TaskSet>> task_cache;
};

namespace cute {

// host planner (plan.cpp)
struct Plan {
  int kind = 0;
  int n0 = 0, n1 = 1;
  int slots1 = 1, nslots = 0;
  int R = 1;
  float eps_main = 0;               // R_MU: mu bound of the mu table
  AxisPlan ax[2];
  std::vector<uint32_t> lut;        // all axes
  std::vector<float> band;          // (lo, hi) per edge per axis
  std::vector<float> mu_eps;        // per r slot
  std::vector<float> mu_edge;       // FP32 mu edges
  std::vector<double> E0, E1;       // FP64 squared edges
  // device copies
  uint32_t *d_lut = nullptr;
  float *d_band = nullptr, *d_mu_eps = nullptr, *d_mu_edge = nullptr;
  double *d_E0 = nullptr, *d_E1 = nullptr;
  ~Plan();
};

struct ErrorParams {
  double eta0;      // per-component absolute FP32 error bound, without the |delta| term
  double eta_l;     // R_MU: absolute error bound of the line-of-sight vector
  double lmin;      // R_MU: lower bound of |l| for pairs within reach
};

// Build the binning plan.  hist_budget_bytes: per-warp histogram budget.
std::string plan_build(int kind, const double *e0, int n0, const double *e1, int n1,
                       const ErrorParams &ep, int lut_budget_words, size_t hist_budget_bytes,
                       Plan &out);

// Task list for one pair set of catalogs on a shared geometry.
void tasks_build(const Geometry &g, const std::vector<int32_t> &csA,
                 const std::vector<int32_t> &csB, bool is_auto, int pair_index, int home_chunk,
                 int slice, bool full_stencil, std::vector<Task> &out,
                 unsigned long long &candidates);

}  // namespace cute

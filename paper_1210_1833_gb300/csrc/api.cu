// api.cu -- the C ABI of libcute_gb.so (include/cute.h): contexts, catalogs,
// cell grids and the counting driver.  The driver validates a request,
// derives the FP32 error bounds from the catalog geometry, builds (or reuses)
// the binning plan and the work list, launches the persistent counting
// kernel and copies the histograms out.
#include "cute_internal.h"
#include "df_stage.h"
#include "count_kernel.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <sstream>

namespace cute {
cute_status catalog_stage(cute_ctx *ctx, Catalog &c, const double *xyz, const float *w);
void catalog_release(cute_ctx *ctx, Catalog &c);
cute_status grid_build(cute_ctx *ctx, const std::vector<Catalog *> &cats, const double reach[3],
                       int kreq);
cute_status ensure_scratch(cute_ctx *ctx, size_t bytes);
cudaError_t launch_count_mono(const KParams &p, bool periodic, int acc, int hp, int blocks,
                              int threads, size_t smem, cudaStream_t st);
cudaError_t launch_count_sigpi(const KParams &p, bool periodic, int acc, int hp, int blocks,
                               int threads, size_t smem, cudaStream_t st);
cudaError_t launch_count_rmu(const KParams &p, int acc, int hp, int blocks, int threads,
                             size_t smem, cudaStream_t st);
}  // namespace cute

using namespace cute;

static thread_local std::string g_create_err;

static cute_status fail(cute_ctx *ctx, cute_status st, const std::string &m) {
  if (ctx) ctx->err = m;
  else g_create_err = m;
  return st;
}

#define CUDA_OR_FAIL(call)                                                         \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? CUTE_E_OOM : CUTE_E_CUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

#define ENTER(ctx)                                                      \
  do {                                                                  \
    if (!(ctx)) return CUTE_E_INVALID;                                  \
    (ctx)->err.clear();                                                 \
    cudaError_t e0_ = cudaSetDevice((ctx)->device);                     \
    if (e0_ != cudaSuccess) return fail(ctx, CUTE_E_CUDA, cudaGetErrorString(e0_)); \
  } while (0)

static bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

extern "C" {

const char *cute_version(void) { return "cute_gb 0.1 (sm_103a)"; }

cute_status cute_ctx_create(int device, void *cuda_stream, cute_ctx **out) {
  if (!out) return fail(nullptr, CUTE_E_INVALID, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(nullptr, CUTE_E_CUDA, "no CUDA device available");
  }
  if (device < 0 || device >= ndev) return fail(nullptr, CUTE_E_INVALID, "bad device index");
  if (cudaSetDevice(device) != cudaSuccess) return fail(nullptr, CUTE_E_CUDA, "cudaSetDevice failed");
  cute_ctx *ctx = new (std::nothrow) cute_ctx();
  if (!ctx) return fail(nullptr, CUTE_E_OOM, "host allocation failed");
  ctx->device = device;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete ctx;
    return fail(nullptr, CUTE_E_CUDA, "cudaGetDeviceProperties failed");
  }
  ctx->sm_count = prop.multiProcessorCount;
  ctx->smem_optin = prop.sharedMemPerBlockOptin;
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return fail(nullptr, CUTE_E_CUDA, "cudaStreamCreate failed");
    }
    ctx->own_stream = true;
  }
  cudaMemPoolProps pp;
  std::memset(&pp, 0, sizeof(pp));
  pp.allocType = cudaMemAllocationTypePinned;
  pp.location.type = cudaMemLocationTypeDevice;
  pp.location.id = device;
  uint64_t keep = UINT64_MAX;  // never trim the pool between requests
  if (cudaMemPoolCreate(&ctx->pool, &pp) != cudaSuccess ||
      cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
    cudaGetLastError();
    ctx->pool = nullptr;
    cute_ctx_destroy(ctx);
    return fail(nullptr, CUTE_E_UNSUPPORTED, "stream-ordered memory pools are not available");
  }
  if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&ctx->d_ticket, 8 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess ||
      cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess) {
    cudaGetLastError();
    cute_ctx_destroy(ctx);
    return fail(nullptr, CUTE_E_OOM, "context allocation failed");
  }
  *out = ctx;
  return CUTE_OK;
}

cute_status cute_ctx_destroy(cute_ctx *ctx) {
  if (!ctx) return CUTE_OK;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  ctx->plans.clear();
  ctx->clear_caches();
  for (auto &kv : ctx->cats) catalog_release(ctx, kv.second);
  ctx->cats.clear();
  cudaFree(ctx->d_ticket);
  cudaFree(ctx->d_err);
  cudaFree(ctx->d_scratch);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);  // pool blocks returned
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  for (auto &kv : ctx->pinned_free) cudaFreeHost(kv.second);
  ctx->pinned_free.clear();
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  cudaGetLastError();
  delete ctx;
  return CUTE_OK;
}

const char *cute_last_error(const cute_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

cute_status cute_sync(cute_ctx *ctx) {
  ENTER(ctx);
  CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream));
  int err = 0;
  CUDA_OR_FAIL(cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    CUDA_OR_FAIL(cudaMemset(ctx->d_err, 0, sizeof(int)));
    return fail(ctx, (cute_status)err, "a kernel reported an error");
  }
  return CUTE_OK;
}

cute_status cute_catalog_upload(cute_ctx *ctx, const double *xyz, const float *w, int64_t n,
                                cute_boundary boundary, double box_L, int32_t *cat_id) {
  ENTER(ctx);
  if (!cat_id) return fail(ctx, CUTE_E_INVALID, "cat_id is NULL");
  if (n < 0 || n > 0x7fffffffLL) return fail(ctx, CUTE_E_INVALID, "n out of range");
  if (n > 0 && !xyz) return fail(ctx, CUTE_E_INVALID, "xyz is NULL");
  if (boundary != CUTE_PERIODIC && boundary != CUTE_OPEN)
    return fail(ctx, CUTE_E_INVALID, "bad boundary");
  if (boundary == CUTE_PERIODIC && !(box_L > 0 && std::isfinite(box_L)))
    return fail(ctx, CUTE_E_INVALID, "periodic catalogs need box_L > 0");
  Catalog c;
  c.id = ctx->next_cat++;
  c.n = n;
  c.boundary = boundary;
  c.L = boundary == CUTE_PERIODIC ? box_L : 0.0;
  cute_status st = catalog_stage(ctx, c, xyz, w);
  if (st != CUTE_OK) {
    std::string m = ctx->err;
    catalog_release(ctx, c);
    return fail(ctx, st, m);
  }
  ctx->cats[c.id] = c;
  *cat_id = c.id;
  return CUTE_OK;
}

cute_status cute_catalog_free(cute_ctx *ctx, int32_t cat_id) {
  ENTER(ctx);
  auto it = ctx->cats.find(cat_id);
  if (it == ctx->cats.end()) return fail(ctx, CUTE_E_STATE, "unknown catalog");
  CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream));
  ctx->clear_caches();
  catalog_release(ctx, it->second);
  ctx->cats.erase(it);
  return CUTE_OK;
}

cute_status cute_catalog_size(cute_ctx *ctx, int32_t cat_id, int64_t *n) {
  ENTER(ctx);
  auto it = ctx->cats.find(cat_id);
  if (it == ctx->cats.end() || !n) return fail(ctx, CUTE_E_STATE, "unknown catalog");
  *n = it->second.n;
  return CUTE_OK;
}

cute_status cute_grid_build(cute_ctx *ctx, const int32_t *cat_ids, int32_t n_cats,
                            const double reach[3], int32_t cells_per_reach) {
  ENTER(ctx);
  if (!cat_ids || n_cats < 1 || !reach) return fail(ctx, CUTE_E_INVALID, "bad arguments");
  if (cells_per_reach < 0 || cells_per_reach > 8)
    return fail(ctx, CUTE_E_INVALID, "cells_per_reach must be 1..8, or 0");
  for (int k = 0; k < 3; k++)
    if (!(reach[k] > 0) || !std::isfinite(reach[k])) return fail(ctx, CUTE_E_INVALID, "reach must be > 0");
  std::vector<Catalog *> cats;
  for (int i = 0; i < n_cats; i++) {
    auto it = ctx->cats.find(cat_ids[i]);
    if (it == ctx->cats.end()) return fail(ctx, CUTE_E_STATE, "unknown catalog");
    for (Catalog *c : cats)
      if (c == &it->second) return fail(ctx, CUTE_E_INVALID, "catalog listed twice");
    cats.push_back(&it->second);
  }
  if (cells_per_reach == 0) {
    // from the mean number of objects in a reach-sized box: dense catalogs
    // gain from finer cells (the candidate volume tightens around the
    // reach), sparse ones lose (every home chunk then spans more cells)
    double per_box = 0;
    for (Catalog *c : cats) {
      double vol = 1.0;
      for (int k = 0; k < 3; k++)
        vol *= c->boundary == CUTE_PERIODIC ? c->L : std::max(c->hi[k] - c->lo[k], reach[k]);
      if (c->n > 0) per_box = std::max(per_box, (double)c->n / vol * reach[0] * reach[1] * reach[2]);
    }
    cells_per_reach = per_box < 600.0 ? 2 : (per_box < 3000.0 ? 3 : 4);
  }
  for (Catalog *c : cats) {
    if (c->boundary != cats[0]->boundary || c->L != cats[0]->L)
      return fail(ctx, CUTE_E_INVALID, "catalogs of one grid must share boundary and box");
  }
  CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream));
  ctx->clear_caches();
  return grid_build(ctx, cats, reach, cells_per_reach);
}

cute_status cute_set_timing(cute_ctx *ctx, int32_t on) {
  ENTER(ctx);
  ctx->timing = on != 0;
  return CUTE_OK;
}

cute_status cute_set_launch(cute_ctx *ctx, int32_t hp, int32_t warps, int32_t slice,
                            int32_t table_binning) {
  ENTER(ctx);
  if (hp != 0 && hp != 2 && hp != 4) return fail(ctx, CUTE_E_INVALID, "home_per_lane must be 0, 2 or 4");
  if (warps < 0 || warps > 20) return fail(ctx, CUTE_E_INVALID, "warps_per_block must be 0..20");
  if (slice < 0 || slice % kTile) return fail(ctx, CUTE_E_INVALID, "slice must be a multiple of 64");
  ctx->hp_override = hp;
  ctx->warps_override = warps;
  ctx->slice_override = slice;
  ctx->table_binning = table_binning != 0;
  return CUTE_OK;
}

cute_status cute_last_stats(cute_ctx *ctx, cute_stats *out) {
  ENTER(ctx);
  if (!out) return fail(ctx, CUTE_E_INVALID, "out is NULL");
  CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream));
  unsigned long long h[kCounterWords] = {0};
  CUDA_OR_FAIL(cudaMemcpy(h, ctx->d_ticket, sizeof(h), cudaMemcpyDeviceToHost));
  ctx->stats.rechecked_pairs = h[1];
  ctx->stats.fp64_pairs = h[6];
  ctx->stats.work_items = h[2];
  ctx->stats.pair_slots = h[4];
  ctx->stats.candidate_pairs = h[5];
  if (ctx->timing && ctx->stats.launches > 0) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1) == cudaSuccess) ctx->stats.kernel_ms = ms;
    cudaGetLastError();
  }
  *out = ctx->stats;
  return CUTE_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ count driver
namespace cute {

// Objects per reach-length of an occupied row of cells: 128-object home
// chunks (4 per lane) pay off where rows are dense enough that a chunk spans
// little more than the cells a 64-object chunk would.
double row_density(const Catalog &A, const Geometry &g) {
  return A.occupied_cells > 0 ? (double)A.n / (double)A.occupied_cells * g.k[0] : 0.0;
}

cute_status validate_desc(cute_ctx *ctx, const cute_pair_desc *d, DescInfo &di) {
  if (!d) return fail(ctx, CUTE_E_INVALID, "descriptor is NULL");
  if (d->kind < CUTE_MONO || d->kind > CUTE_THETA) return fail(ctx, CUTE_E_INVALID, "bad kind");
  const bool two_d = (d->kind == CUTE_R_MU || d->kind == CUTE_SIGMA_PI);
  if (!d->edges0 || d->n0 < 1 || d->n0 > 4096) return fail(ctx, CUTE_E_INVALID, "edges0/n0 invalid");
  if (two_d && (!d->edges1 || d->n1 < 1 || d->n1 > 4096)) return fail(ctx, CUTE_E_INVALID, "edges1/n1 invalid");
  for (int k = 0; k <= d->n0; k++) {
    if (!(d->edges0[k] >= 0) || !std::isfinite(d->edges0[k]) || (k && !(d->edges0[k] > d->edges0[k - 1])))
      return fail(ctx, CUTE_E_INVALID, "edges0 must be finite, >= 0 and strictly increasing");
  }
  if (two_d) {
    for (int k = 0; k <= d->n1; k++) {
      if (!(d->edges1[k] >= 0) || !std::isfinite(d->edges1[k]) ||
          (k && !(d->edges1[k] > d->edges1[k - 1])))
        return fail(ctx, CUTE_E_INVALID, "edges1 must be finite, >= 0 and strictly increasing");
    }
    if (d->kind == CUTE_R_MU && (d->edges1[0] != 0.0 || d->edges1[d->n1] != 1.0))
      return fail(ctx, CUTE_E_INVALID, "mu edges must run from 0 to 1");
  }
  auto ia = ctx->cats.find(d->cat_a), ib = ctx->cats.find(d->cat_b);
  if (ia == ctx->cats.end() || ib == ctx->cats.end()) return fail(ctx, CUTE_E_STATE, "unknown catalog");
  di.A = &ia->second;
  di.B = &ib->second;
  di.is_auto = (d->cat_a == d->cat_b);
  di.kind = (int)d->kind;
  if (di.A->geom < 0 || di.B->geom < 0) return fail(ctx, CUTE_E_STATE, "catalog has no cell grid");
  if (di.A->geom != di.B->geom) return fail(ctx, CUTE_E_STATE, "catalogs are on different grids");
  auto gi = ctx->geoms.find(di.A->geom);
  if (gi == ctx->geoms.end()) return fail(ctx, CUTE_E_STATE, "grid geometry missing");
  di.g = &gi->second;
  if ((d->kind == CUTE_R_MU || d->kind == CUTE_THETA) && di.g->periodic)
    return fail(ctx, CUTE_E_UNSUPPORTED, "R_MU and THETA are defined for open catalogs only");
  double r0 = d->edges0[d->n0];
  if (d->kind == CUTE_SIGMA_PI) {
    di.need[0] = di.need[1] = r0;
    di.need[2] = d->edges1[d->n1];
  } else {
    di.need[0] = di.need[1] = di.need[2] = r0;
  }
  for (int k = 0; k < 3; k++)
    if (di.need[k] > di.g->reach[k])
      return fail(ctx, CUTE_E_STATE, "the grid's reach is smaller than the largest edge");
  if (d->weighted && (!di.A->d_w || !di.B->d_w) && (di.A->n > 0 && di.B->n > 0))
    return fail(ctx, CUTE_E_STATE, "weighted counts need catalogs uploaded with weights");
  return CUTE_OK;
}

static const double kU32 = 5.9604644775390625e-08;

// largest separation component that can decide a bin: the top edge of r,
// chord or sigma, and of pi
double decision_reach(const cute_pair_desc *d) {
  double r = d->edges0[d->n0];
  if (d->kind == CUTE_SIGMA_PI) r = std::max(r, d->edges1[d->n1]);
  return r;
}

cudaError_t dev_alloc(cute_ctx *ctx, void **p, size_t bytes) {
  return cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), ctx->pool, ctx->stream);
}
void dev_free(cute_ctx *ctx, void *p) {
  if (p) cudaFreeAsync(p, ctx->stream);
}
cudaError_t pinned_get(cute_ctx *ctx, size_t n, int32_t **p, size_t *cap) {
  auto it = ctx->pinned_free.lower_bound(n);
  if (it != ctx->pinned_free.end()) {
    *cap = it->first;
    *p = it->second;
    ctx->pinned_free.erase(it);
    return cudaSuccess;
  }
  const size_t c = n + n / 4 + 16;
  cudaError_t e = cudaMallocHost((void **)p, c * sizeof(int32_t));
  if (e == cudaSuccess) *cap = c;
  return e;
}
void pinned_put(cute_ctx *ctx, int32_t *p, size_t cap) {
  if (p) ctx->pinned_free.emplace(cap, p);
}

// The double-float view of a pair set: remainders, and the error bounds of
// its separation and line-of-sight components (df_stage.h).
PairDF pair_df(const DescInfo &di) {
  const Geometry &g = *di.g;
  PairDF f;
  std::memset(&f, 0, sizeof(f));
  f.loA = di.A->d_lo;
  f.loB = di.B->d_lo;
  double xm = std::max(g.xmax[0], std::max(g.xmax[1], g.xmax[2]));
  double fom = std::max(std::fabs(g.fo[0]), std::max(std::fabs(g.fo[1]), std::fabs(g.fo[2])));
  double am = std::max(g.absmax[0], std::max(g.absmax[1], g.absmax[2]));
  const double Lp = g.periodic ? g.L : 0.0;
  f.eta = (float)dfs::eta_sep(xm, Lp);
  f.eta_l = (float)dfs::eta_los(xm, fom, am);
  if (g.periodic) {
    f.Lh = (float)g.L;
    f.Ll = (float)(g.L - (double)f.Lh);
  }
  for (int k = 0; k < 3; k++) {
    const double t = 2.0 * g.fo[k];
    f.fo2h[k] = (float)t;
    f.fo2l[k] = (float)(t - (double)f.fo2h[k]);
  }
  return f;
}

PairDev pair_dev(const DescInfo &di, int out) {
  PairDev pd;
  std::memset(&pd, 0, sizeof(pd));
  pd.posA = di.A->d_pos;
  pd.posB = di.B->d_pos;
  pd.qA = di.A->d_posq;
  pd.qB = di.B->d_posq;
  pd.q0 = di.g->q0;
  pd.sA = di.A->d_s64;
  pd.sB = di.B->d_s64;
  pd.permA = di.A->d_perm;
  pd.nA = (int32_t)di.A->n;
  pd.nB = (int32_t)di.B->n;
  pd.out = (int32_t)out;
  pd.is_auto = di.is_auto;
  pd.L32 = (float)di.g->L;
  pd.L64 = di.g->periodic ? di.g->L : 0.0;
  return pd;
}

ErrorParams error_params(const std::vector<DescInfo> &dis, double rmax) {
  ErrorParams ep{0, 0, 0, 0, 0};
  double rmin = 1e300;
  for (const DescInfo &di : dis) {
    const Geometry &g = *di.g;
    double xm = std::max(g.xmax[0], std::max(g.xmax[1], g.xmax[2]));
    double e;
    if (g.periodic) {
      // per component of d = q - (a - S): FP32 frame offsets of both objects
      // (|q|, |a| <= xm), the home's image a - S (|a - S| <= |q| + |d|, and
      // only |d| up to the reach decides a bin), the FP32 box size L32 = S
      const double dL = std::fabs((double)(float)g.L - g.L);
      e = kU32 * (3.0 * xm + 2.0 * rmax) * 1.01 + dL * 1.01 + 1e-12 * (xm + g.L);
    } else {
      e = kU32 * 2.0 * xm * 1.01 + 1e-12 * xm;
    }
    ep.eta0 = std::max(ep.eta0, e);
    ep.xm = std::max(ep.xm, xm);
    rmin = std::min(rmin, g.rmin);
    ep.qd = std::max(ep.qd, g.qd);
    ep.q0 = std::max(ep.q0, g.q0);
  }
  ep.lmin = 2.0 * rmin - rmax;
  return ep;
}

// Per-warp budget of the count histogram's copies: plain counts take as
// many copies (<= 32) as fit in 12 KB (fewer bank conflicts), 4 KB for the
// kernel that runs 20 warps (plain monopole / theta, two home objects per
// lane) so that 20 warps fit beside the binning tables; weighted counts,
// whose 32 float-float columns already take most of a warp's shared memory
// and whose per-pair cost is the column update, keep about 1 KB so that
// more warps fit.
size_t hist_budget(const cute_pair_desc *d, int acc, int hp) {
  const bool two_d = (d->kind == CUTE_R_MU || d->kind == CUTE_SIGMA_PI);
  const size_t nslots = (size_t)(d->n0 + 2) * (two_d ? (size_t)(d->n1 + 2) : 1u);
  size_t want = 12288;
  if (acc == 1) want = 1024;
  else if (acc == 0 && count_max_warps(!two_d, hp, acc) > 16) want = 4096;
  // integer weights: two histograms (counts, weight products) in the same 4 KB
  else if (acc == 3) want = count_max_warps(!two_d, hp, acc) > 16 ? 2048 : 6144;
  return std::min<size_t>(12288, std::max<size_t>(want, nslots * 4));
}

cute_status get_plan(cute_ctx *ctx, const cute_pair_desc *d, const ErrorParams &ep, int hp,
                     int acc, std::shared_ptr<Plan> &out) {
  std::ostringstream key;
  key.precision(17);
  const size_t hb = hist_budget(d, acc, hp);
  key << d->kind << "|" << ep.eta0 << "|" << ep.lmin << "|" << ep.xm << "|" << ep.qd << "|"
      << ep.q0 << "|" << hp << "|"
      << ctx->table_binning << "|" << hb << "|";
  for (int k = 0; k <= d->n0; k++) key << d->edges0[k] << ",";
  if (d->kind == CUTE_R_MU || d->kind == CUTE_SIGMA_PI)
    for (int k = 0; k <= d->n1; k++) key << d->edges1[k] << ",";
  auto it = ctx->plans.find(key.str());
  if (it != ctx->plans.end()) {
    out = it->second;
    return CUTE_OK;
  }
  auto P = std::make_shared<Plan>();
  const bool two_d = (d->kind == CUTE_R_MU || d->kind == CUTE_SIGMA_PI);
  std::string m = plan_build((int)d->kind, d->edges0, d->n0, d->edges1, two_d ? d->n1 : 1, ep,
                             two_d ? 8192 : 8192, hb, !ctx->table_binning, *P);
  if (!m.empty()) return fail(ctx, CUTE_E_UNSUPPORTED, m);
  auto up = [&](void **dst, const void *src, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  CUDA_OR_FAIL(up((void **)&P->d_lut, P->lut.data(), P->lut.size() * 4));
  CUDA_OR_FAIL(up((void **)&P->d_band, P->band.data(), P->band.size() * 4));
  CUDA_OR_FAIL(up((void **)&P->d_E0, P->E0.data(), P->E0.size() * 8));
  CUDA_OR_FAIL(up((void **)&P->d_E1, P->E1.data(), P->E1.size() * 8));
  CUDA_OR_FAIL(up((void **)&P->d_E0df, P->E0df.data(), P->E0df.size() * 4));
  CUDA_OR_FAIL(up((void **)&P->d_E1df, P->E1df.data(), P->E1df.size() * 4));
  ctx->plans[key.str()] = P;
  out = P;
  return CUTE_OK;
}

cute_status get_work(cute_ctx *ctx, const std::vector<DescInfo> &dis, int hp, int slice,
                      bool full_stencil, std::shared_ptr<WorkSet> &out) {
  std::ostringstream key;
  key.precision(17);
  key << hp << "|" << slice << "|" << full_stencil << "|";
  for (const DescInfo &di : dis)
    key << di.A->id << ":" << di.A->grid_version << ":" << di.B->id << ":" << di.B->grid_version
        << ":" << di.kind << ":" << di.need[0] << ":" << di.need[1] << ":" << di.need[2] << ",";
  auto it = ctx->work_cache.find(key.str());
  if (it != ctx->work_cache.end()) {
    out = it->second;
    return CUTE_OK;
  }
  if (dis.size() > 65536) return fail(ctx, CUTE_E_UNSUPPORTED, "more than 65536 pair sets");
  auto T = std::make_shared<WorkSet>();
  const int home_chunk = 32 * hp;
  std::vector<std::vector<int4>> chunks(dis.size()), stencils(dis.size());
  size_t nch = 0, nst = 0;
  T->ebase.assign(1, 0);
  long long entries = 0;
  for (size_t i = 0; i < dis.size(); i++) {
    const DescInfo &di = dis[i];
    if (di.A->n > 0 && di.B->n > 0) {
      const int shape = (di.kind == CUTE_SIGMA_PI) ? kShapeDiskSlab : kShapeBall;
      auto ci = di.A->chunk_cache.find(home_chunk);
      if (ci == di.A->chunk_cache.end()) {
        ci = di.A->chunk_cache.emplace(home_chunk, std::vector<int4>()).first;
        chunks_build(*di.g, di.A->h_cell_start, home_chunk, ci->second);
      }
      chunks[i] = ci->second;
      stencil_build(*di.g, di.is_auto, full_stencil, shape, di.need, stencils[i]);
    }
    nch += chunks[i].size();
    nst += stencils[i].size();
    entries += (long long)chunks[i].size() * (long long)stencils[i].size();
    if (entries > (1LL << 30)) return fail(ctx, CUTE_E_UNSUPPORTED, "too many work entries");
    T->ebase.push_back((int)entries);
  }
  T->nentries = (int)entries;
  T->st = ctx->stream;
  CUDA_OR_FAIL(dev_alloc(ctx, (void **)&T->d_chunks, std::max<size_t>(nch, 1) * sizeof(int4)));
  CUDA_OR_FAIL(dev_alloc(ctx, (void **)&T->d_pdf, dis.size() * sizeof(PairDF)));
  CUDA_OR_FAIL(dev_alloc(ctx, (void **)&T->d_stencil, std::max<size_t>(nst, 1) * sizeof(int4)));
  size_t oc = 0, os = 0;
  for (size_t i = 0; i < dis.size(); i++) {
    const DescInfo &di = dis[i];
    PairDev pd = pair_dev(di, (int)i);
    pd.df = T->d_pdf + i;
    T->pdf.push_back(pair_df(di));
    PairWork pw;
    std::memset(&pw, 0, sizeof(pw));
    pw.chunks = T->d_chunks + oc;
    pw.stencil = T->d_stencil + os;
    pw.csB = di.B->d_cell_start;
    pw.nchunks = (int32_t)chunks[i].size();
    pw.nstencil = std::max<int32_t>(1, (int32_t)stencils[i].size());
    pw.nx = di.g->nc[0];
    pw.ny = di.g->nc[1];
    pw.nz = di.g->nc[2];
    pw.mode = !di.is_auto ? kModeCross : (full_stencil ? kModeAutoFull : kModeAutoHalf);
    pw.periodic = di.g->periodic;
    T->work.push_back(pw);
    T->pairs.push_back(pd);
    if (!chunks[i].empty())
      CUDA_OR_FAIL(cudaMemcpyAsync(T->d_chunks + oc, chunks[i].data(), chunks[i].size() * sizeof(int4),
                                   cudaMemcpyHostToDevice, ctx->stream));
    if (!stencils[i].empty())
      CUDA_OR_FAIL(cudaMemcpyAsync(T->d_stencil + os, stencils[i].data(),
                                   stencils[i].size() * sizeof(int4), cudaMemcpyHostToDevice,
                                   ctx->stream));
    oc += chunks[i].size();
    os += stencils[i].size();
  }
  CUDA_OR_FAIL(cudaMemcpyAsync(T->d_pdf, T->pdf.data(), T->pdf.size() * sizeof(PairDF),
                               cudaMemcpyHostToDevice, ctx->stream));
  CUDA_OR_FAIL(dev_alloc(ctx, (void **)&T->d_pairs, T->pairs.size() * sizeof(PairDev)));
  CUDA_OR_FAIL(cudaMemcpyAsync(T->d_pairs, T->pairs.data(), T->pairs.size() * sizeof(PairDev),
                               cudaMemcpyHostToDevice, ctx->stream));
  CUDA_OR_FAIL(dev_alloc(ctx, (void **)&T->d_work, T->work.size() * sizeof(PairWork)));
  CUDA_OR_FAIL(cudaMemcpyAsync(T->d_work, T->work.data(), T->work.size() * sizeof(PairWork),
                               cudaMemcpyHostToDevice, ctx->stream));
  CUDA_OR_FAIL(dev_alloc(ctx, (void **)&T->d_ebase, T->ebase.size() * sizeof(int)));
  CUDA_OR_FAIL(cudaMemcpyAsync(T->d_ebase, T->ebase.data(), T->ebase.size() * sizeof(int),
                               cudaMemcpyHostToDevice, ctx->stream));
  CUDA_OR_FAIL(dev_alloc(ctx, (void **)&T->d_cnt, std::max(T->nentries, 1) * sizeof(int)));
  CUDA_OR_FAIL(dev_alloc(ctx, (void **)&T->d_bsum, work_bsum_words(T->nentries) * sizeof(long long)));
  CUDA_OR_FAIL(dev_alloc(ctx, (void **)&T->d_eprefix, (T->nentries + 1) * sizeof(long long)));
  CUDA_OR_FAIL(dev_alloc(ctx, (void **)&T->d_spairs, sizeof(unsigned long long)));
  CUDA_OR_FAIL(work_count(T->d_work, T->d_ebase, (int)T->pairs.size(), T->nentries, slice,
                          T->d_cnt, T->d_bsum, T->d_eprefix, T->d_spairs, ctx->stream));
  // the item count sizes the record list: one round trip per work list
  CUDA_OR_FAIL(cudaMemcpyAsync(&T->items, T->d_eprefix + T->nentries, sizeof(long long),
                               cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_OR_FAIL(cudaMemcpyAsync(&T->stencil_pairs, T->d_spairs, sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream));
  CUDA_OR_FAIL(dev_alloc(ctx, (void **)&T->d_items, std::max<long long>(T->items, 1) * sizeof(int4)));
  CUDA_OR_FAIL(work_write(T->d_work, T->d_ebase, (int)T->pairs.size(), T->nentries, slice,
                          T->d_eprefix, T->d_items, ctx->stream));
  ctx->work_cache[key.str()] = T;
  out = T;
  return CUTE_OK;
}

// identity of a request for the autotuner's memory: kind, catalogs (and
// their grid versions), accumulation policy, stencil
std::string tuning_key(const std::vector<DescInfo> &dis, int acc, bool full_stencil) {
  // by problem shape (kind, sizes, cell grid), so re-uploaded catalogs of
  // the same workload keep their tuning
  std::ostringstream k;
  k << (acc == 3 ? 1 : acc) << "|" << full_stencil << "|";  // integer weights: a weighted count
  for (const DescInfo &di : dis)
    k << di.kind << ":" << di.is_auto << ":" << di.A->n << ":" << di.B->n << ":" << di.g->nc[0]
      << "x" << di.g->nc[1] << "x" << di.g->nc[2] << ",";
  return k.str();
}

// common preparation of a (batched) count: validation, plan, work list, params
struct Prepared {
  std::vector<DescInfo> dis;
  std::shared_ptr<Plan> plan;
  std::shared_ptr<WorkSet> ts;
  KParams p;
  int hp, warps, blocks, acc;
  size_t smem;
};

cute_status prepare(cute_ctx *ctx, int n, const cute_pair_desc *d, int acc, bool full_stencil,
                    Prepared &pr, bool allow_swap = true) {
  if (n < 1 || !d) return fail(ctx, CUTE_E_INVALID, "no descriptors");
  pr.dis.resize(n);
  for (int i = 0; i < n; i++) {
    cute_status st = validate_desc(ctx, &d[i], pr.dis[i]);
    if (st != CUTE_OK) return st;
    // every separation measure is symmetric in the pair (bit for bit: the
    // canonical separation only changes sign), so a cross count may put the
    // larger catalog on the home side, where fuller cells fill the lanes
    if (allow_swap && !pr.dis[i].is_auto && pr.dis[i].B->n > pr.dis[i].A->n)
      std::swap(pr.dis[i].A, pr.dis[i].B);
    if (i > 0) {
      bool same = d[i].kind == d[0].kind && d[i].n0 == d[0].n0 && d[i].weighted == d[0].weighted &&
                  std::equal(d[i].edges0, d[i].edges0 + d[i].n0 + 1, d[0].edges0);
      if (same && (d[0].kind == CUTE_R_MU || d[0].kind == CUTE_SIGMA_PI))
        same = d[i].n1 == d[0].n1 && std::equal(d[i].edges1, d[i].edges1 + d[i].n1 + 1, d[0].edges1);
      if (!same) return fail(ctx, CUTE_E_INVALID, "batched descriptors must share kind, edges and weighted");
      if (pr.dis[i].g->periodic != pr.dis[0].g->periodic)
        return fail(ctx, CUTE_E_INVALID, "batched descriptors must share the boundary");
    }
  }
  ErrorParams ep = error_params(pr.dis, decision_reach(&d[0]));
  // weighted monopole / chord counts whose catalogs hold integer weights in
  // [0, 2048] (counts per pixel or cell) sum the weight products in integer
  // histograms: exact, and without the float-float columns
  unsigned wpmax = 0;
  if (acc == 1 && (d[0].kind == CUTE_MONO || d[0].kind == CUTE_THETA)) {
    bool ints = true;
    for (const DescInfo &di : pr.dis) {
      if (di.A->wint < 0 || di.B->wint < 0) ints = false;
      else wpmax = std::max(wpmax, (unsigned)di.A->wint * (unsigned)di.B->wint);
    }
    if (ints) acc = 3;
  }
  // home objects per lane: 4 when home cells hold enough objects to fill
  // 128-object chunks, else 2
  pr.hp = ctx->hp_override;
  if (!pr.hp) {
    // object-weighted mean over the pair sets of a batch
    double dens = 0, objs = 0;
    for (const DescInfo &di : pr.dis) {
      dens += (double)di.A->n * row_density(*di.A, *di.g);
      objs += (double)di.A->n;
    }
    pr.hp = (objs > 0 && dens / objs >= 2000.0) ? 4 : 2;
    // plain monopole / theta counts: the two-per-lane kernel runs 20 warps,
    // which outweighs the denser rows' case for four (c3 DD: 3.20 s against
    // 3.32 s)
    if ((acc == 0 || acc == 3) && (d[0].kind == CUTE_MONO || d[0].kind == CUTE_THETA)) pr.hp = 2;
  }
  int slice = ctx->slice_override ? ctx->slice_override : 2048;
  int warps_tuned = 0;
  {
    auto it = ctx->tuned.find(tuning_key(pr.dis, acc, full_stencil));
    if (it != ctx->tuned.end()) {
      if (!ctx->hp_override) pr.hp = it->second.home_per_lane;
      if (!ctx->slice_override) slice = it->second.slice;
      warps_tuned = it->second.warps_per_block;
    }
  }
  if (acc == 3) {
    // one item adds at most 2 (32 / R) HP slice products to a weight-sum copy
    // (R >= 1): the slice keeps that below 2^32, else float-float columns
    const unsigned long long per = 2ull * 32 * (unsigned long long)pr.hp * std::max(wpmax, 1u);
    const long long smax = (long long)(0xFFFFFFFFull / per) / kTile * kTile;
    if (smax < kTile) acc = 1;
    else slice = (int)std::min<long long>(slice, smax);
  }
  cute_status st = get_plan(ctx, &d[0], ep, pr.hp, acc, pr.plan);
  if (st != CUTE_OK) return st;
  st = get_work(ctx, pr.dis, pr.hp, slice, full_stencil, pr.ts);
  if (st != CUTE_OK) return st;
  const Plan &P = *pr.plan;
  SmemLayout L = smem_layout((int)P.lut.size(), (int)P.band.size() / 2, P.nslots, P.R, pr.hp, acc,
                             d[0].kind == CUTE_R_MU && acc != 0,
                             d[0].kind == CUTE_R_MU || acc != 0);
  pr.acc = acc;
  size_t avail = ctx->smem_optin;
  const int wmax = count_max_warps(d[0].kind == CUTE_MONO || d[0].kind == CUTE_THETA, pr.hp, acc);
  int warps = ctx->warps_override ? ctx->warps_override : (warps_tuned ? warps_tuned : wmax);
  warps = std::min(warps, wmax);
  while (warps > 1 && (size_t)L.lut_bytes + (size_t)warps * L.warp_bytes > avail) warps--;
  if ((size_t)L.lut_bytes + (size_t)warps * L.warp_bytes > avail)
    return fail(ctx, CUTE_E_UNSUPPORTED,
                acc == 1 ? "too many bins for weighted counts (32 float-float columns per warp)"
                         : "binning tables do not fit in shared memory");
  pr.warps = warps;
  pr.smem = (size_t)L.lut_bytes + (size_t)warps * L.warp_bytes;
  pr.blocks = ctx->sm_count;
  KParams &p = pr.p;
  std::memset(&p, 0, sizeof(p));
  p.items = pr.ts->d_items;
  p.total = pr.ts->items;
  p.item_stride = 1;
  p.pairs = pr.ts->d_pairs;
  p.lut = P.d_lut;
  p.lut_words = (int)P.lut.size();
  p.ax[0] = P.ax[0];
  p.ax[1] = P.ax[1];
  p.band = (const float2 *)P.d_band;
  p.band_words = (int)P.band.size() / 2;
  p.mu_eps_base = P.mu_eps_base;
  p.far = P.far;
  p.wpmax = wpmax;
  cull_params(pr.dis, d, n, p);
  p.E0 = P.d_E0;
  p.E1 = P.d_E1;
  p.E0df = (const float2 *)P.d_E0df;
  p.E1df = (const float2 *)P.d_E1df;
  p.n0 = P.n0;
  p.n1 = P.n1;
  p.slots1 = P.slots1;
  p.nslots = P.nslots;
  p.R = P.R;
  p.slice = slice;
  p.ticket = ctx->d_ticket;
  p.stats = ctx->d_ticket + 1;
  p.err = ctx->d_err;
  return CUTE_OK;
}

cudaError_t launch_prepared(cute_ctx *ctx, const Prepared &pr, int kind,
                            cudaStream_t stream = nullptr) {
  const bool per = pr.dis[0].g->periodic;
  const int threads = pr.warps * 32;
  cudaStream_t st = stream ? stream : ctx->stream;
  switch (kind) {
    case CUTE_MONO:
      return launch_count_mono(pr.p, per, pr.acc, pr.hp, pr.blocks, threads, pr.smem, st);
    case CUTE_THETA:
      return launch_count_mono(pr.p, false, pr.acc, pr.hp, pr.blocks, threads, pr.smem, st);
    case CUTE_SIGMA_PI:
      return launch_count_sigpi(pr.p, per, pr.acc, pr.hp, pr.blocks, threads, pr.smem, st);
    default:
      return launch_count_rmu(pr.p, pr.acc, pr.hp, pr.blocks, threads, pr.smem, st);
  }
}

// Capture the device work of a batched count into a CUDA graph (on the
// private capture stream) and return its executable, or null if capture is
// not possible here (the caller then launches normally).
static cudaGraphExec_t capture_batched(cute_ctx *ctx, const Prepared &pr, int kind, int n, int nb,
                                       bool weighted, unsigned long long *d_out, double *d_ws,
                                       uint64_t *const *counts, double *const *wsum) {
  cudaStream_t cs = ctx->cap_stream;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  bool ok = true;
  ok = ok && cudaMemsetAsync(ctx->d_ticket, 0, kCounterWords * sizeof(unsigned long long), cs) == cudaSuccess;
  ok = ok && cudaMemsetAsync(d_out, 0, sizeof(unsigned long long) * (size_t)nb * n, cs) == cudaSuccess;
  if (weighted) ok = ok && cudaMemsetAsync(d_ws, 0, sizeof(double) * (size_t)nb * n, cs) == cudaSuccess;
  if (ok && pr.p.total > 0) ok = launch_prepared(ctx, pr, kind, cs) == cudaSuccess;
  for (int i = 0; ok && i < n; i++) {
    ok = cudaMemcpyAsync(counts[i], d_out + (size_t)i * nb, sizeof(uint64_t) * nb,
                         cudaMemcpyDeviceToDevice, cs) == cudaSuccess;
    if (ok && weighted)
      ok = cudaMemcpyAsync(wsum[i], d_ws + (size_t)i * nb, sizeof(double) * nb,
                           cudaMemcpyDeviceToDevice, cs) == cudaSuccess;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  cudaGraphExec_t ex = nullptr;
  if (ok && e == cudaSuccess && g) {
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  return ex;
}

// Counts (and weighted sums) of n pair sets into counts[k] / wsum[k] (host
// or device); oor for n == 1.
cute_status count_driver(cute_ctx *ctx, int n, const cute_pair_desc *d, uint64_t *const *counts,
                         double *const *wsum, uint64_t *oor) {
  for (int i = 0; i < n; i++)
    if (!counts || !counts[i]) return fail(ctx, CUTE_E_INVALID, "counts is NULL");
  const bool weighted = d[0].weighted != 0;
  if (weighted)
    for (int i = 0; i < n; i++)
      if (!wsum || !wsum[i]) return fail(ctx, CUTE_E_INVALID, "weighted counts need wsum");
  Prepared pr;
  cute_status st = prepare(ctx, n, d, weighted ? 1 : 0, false, pr);
  if (st != CUTE_OK) return st;
  const int nb = pr.p.n0 * pr.p.n1;
  const size_t cnt_bytes = sizeof(unsigned long long) * (size_t)nb * n;
  const size_t ws_bytes = weighted ? sizeof(double) * (size_t)nb * n : 0;
  st = ensure_scratch(ctx, cnt_bytes + ws_bytes + 256);
  if (st != CUTE_OK) return st;
  unsigned long long *d_out = (unsigned long long *)ctx->d_scratch;
  double *d_ws = weighted ? (double *)((char *)ctx->d_scratch + ((cnt_bytes + 255) & ~(size_t)255)) : nullptr;
  pr.p.out_counts = d_out;
  pr.p.out_wsum = d_ws;
  CUDA_OR_FAIL(cudaMemsetAsync(d_out, 0, cnt_bytes, ctx->stream));
  if (weighted) CUDA_OR_FAIL(cudaMemsetAsync(d_ws, 0, ws_bytes, ctx->stream));
  CUDA_OR_FAIL(cudaMemsetAsync(ctx->d_ticket, 0, kCounterWords * sizeof(unsigned long long), ctx->stream));
  ctx->stats = cute_stats{};
  ctx->stats.warps_per_block = pr.warps;
  ctx->stats.blocks = pr.blocks;
  ctx->stats.home_per_lane = pr.hp;
  ctx->stats.stencil_pairs = pr.ts->stencil_pairs;
  // batched counts into device outputs: replay a captured graph
  bool all_dev = n > 1 && oor == nullptr;
  for (int i = 0; all_dev && i < n; i++)
    all_dev = is_device_ptr(counts[i]) && (!weighted || is_device_ptr(wsum[i]));
  if (all_dev) {
    std::ostringstream gk;
    gk << tuning_key(pr.dis, weighted ? 1 : 0, false) << "|" << (const void *)pr.plan.get() << "|"
       << (const void *)pr.ts.get() << "|" << pr.hp << "|" << pr.warps << "|" << pr.p.slice << "|"
       << (const void *)d_out << "|" << (const void *)d_ws;
    for (int i = 0; i < n; i++) gk << "|" << (const void *)counts[i] << "," << (const void *)(weighted ? wsum[i] : nullptr);
    auto it = ctx->graphs.find(gk.str());
    cudaGraphExec_t ex = (it != ctx->graphs.end()) ? it->second : nullptr;
    if (!ex) {
      CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream));
      ex = capture_batched(ctx, pr, (int)d[0].kind, n, nb, weighted, d_out, d_ws, counts, wsum);
      if (ex) ctx->graphs[gk.str()] = ex;
    }
    if (ex) {
      if (ctx->timing) CUDA_OR_FAIL(cudaEventRecord(ctx->ev0, ctx->stream));
      CUDA_OR_FAIL(cudaGraphLaunch(ex, ctx->stream));
      if (ctx->timing) CUDA_OR_FAIL(cudaEventRecord(ctx->ev1, ctx->stream));
      ctx->stats.launches = pr.p.total > 0 ? 1 : 0;
      return CUTE_OK;
    }
  }
  if (ctx->timing) CUDA_OR_FAIL(cudaEventRecord(ctx->ev0, ctx->stream));
  if (pr.p.total > 0) {
    CUDA_OR_FAIL(launch_prepared(ctx, pr, (int)d[0].kind));
    ctx->stats.launches = 1;
  }
  if (ctx->timing) CUDA_OR_FAIL(cudaEventRecord(ctx->ev1, ctx->stream));
  bool need_sync = (oor != nullptr);
  for (int i = 0; i < n; i++) {
    bool dev = is_device_ptr(counts[i]);
    CUDA_OR_FAIL(cudaMemcpyAsync(counts[i], d_out + (size_t)i * nb, sizeof(uint64_t) * nb,
                                 dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 ctx->stream));
    if (!dev) need_sync = true;
    if (weighted) {
      bool wdev = is_device_ptr(wsum[i]);
      CUDA_OR_FAIL(cudaMemcpyAsync(wsum[i], d_ws + (size_t)i * nb, sizeof(double) * nb,
                                   wdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                   ctx->stream));
      if (!wdev) need_sync = true;
    }
  }
  if (need_sync) {
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream));
    int err = 0;
    CUDA_OR_FAIL(cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
      CUDA_OR_FAIL(cudaMemset(ctx->d_err, 0, sizeof(int)));
      return fail(ctx, (cute_status)err, "the counting kernel reported an error");
    }
  }
  if (oor) {
    std::vector<uint64_t> h(nb);
    CUDA_OR_FAIL(cudaMemcpy(h.data(), d_out, sizeof(uint64_t) * nb, cudaMemcpyDeviceToHost));
    uint64_t s = 0;
    for (uint64_t v : h) s += v;
    uint64_t na = (uint64_t)pr.dis[0].A->n, nbb = (uint64_t)pr.dis[0].B->n;
    uint64_t total = pr.dis[0].is_auto ? (na ? na * (na - 1) / 2 : 0) : na * nbb;
    *oor = total - s;
  }
  return CUTE_OK;
}

// Gradient of sum_b G_b W_b with respect to the weights of one catalog: a
// full-stencil pass with that catalog on the home side.
static cute_status adjoint_pass(cute_ctx *ctx, const cute_pair_desc *d, const double *d_G,
                                double *grad, bool *need_sync) {
  Prepared pr;
  cute_status st = prepare(ctx, 1, d, 2, true, pr, false);
  if (st != CUTE_OK) return st;
  const int64_t nA = pr.dis[0].A->n;
  bool dev = is_device_ptr(grad);
  double *d_grad = grad;
  const size_t gbytes = sizeof(double) * (size_t)std::max<int64_t>(nA, 1);
  if (!dev) {
    st = ensure_scratch(ctx, gbytes + 256);
    if (st != CUTE_OK) return st;
    d_grad = (double *)ctx->d_scratch;
  }
  CUDA_OR_FAIL(cudaMemsetAsync(d_grad, 0, gbytes, ctx->stream));
  // the ticket only: the statistics add up over the passes
  CUDA_OR_FAIL(cudaMemsetAsync(ctx->d_ticket, 0, sizeof(unsigned long long), ctx->stream));
  pr.p.G = d_G;
  pr.p.grad = d_grad;
  ctx->stats.stencil_pairs += pr.ts->stencil_pairs;
  ctx->stats.warps_per_block = pr.warps;
  ctx->stats.blocks = pr.blocks;
  ctx->stats.home_per_lane = pr.hp;
  if (pr.p.total > 0) {
    CUDA_OR_FAIL(launch_prepared(ctx, pr, (int)d->kind));
    ctx->stats.launches++;
  }
  if (!dev && nA > 0) {
    CUDA_OR_FAIL(cudaMemcpyAsync(grad, d_grad, sizeof(double) * (size_t)nA, cudaMemcpyDeviceToHost,
                                 ctx->stream));
    *need_sync = true;
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream));
  }
  return CUTE_OK;
}

cute_status adjoint_driver(cute_ctx *ctx, const cute_pair_desc *d, const double *G,
                           double *grad_a, double *grad_b) {
  if (!d || !G || !grad_a) return fail(ctx, CUTE_E_INVALID, "descriptor, G and grad_a are required");
  DescInfo di;
  cute_status st = validate_desc(ctx, d, di);
  if (st != CUTE_OK) return st;
  if (!di.A->d_w || !di.B->d_w)
    if (di.A->n > 0 && di.B->n > 0)
      return fail(ctx, CUTE_E_STATE, "the adjoint needs catalogs uploaded with weights");
  const int nb = d->n0 * ((d->kind == CUTE_R_MU || d->kind == CUTE_SIGMA_PI) ? d->n1 : 1);
  // G on the device, after the output buffers in the scratch area
  double *d_G = nullptr;
  CUDA_OR_FAIL(cudaMallocAsync((void **)&d_G, sizeof(double) * nb, ctx->stream));
  CUDA_OR_FAIL(cudaMemcpyAsync(d_G, G, sizeof(double) * nb, cudaMemcpyDefault, ctx->stream));
  ctx->stats = cute_stats{};
  CUDA_OR_FAIL(cudaMemsetAsync(ctx->d_ticket, 0, kCounterWords * sizeof(unsigned long long), ctx->stream));
  if (ctx->timing) CUDA_OR_FAIL(cudaEventRecord(ctx->ev0, ctx->stream));
  bool need_sync = false;
  st = adjoint_pass(ctx, d, d_G, grad_a, &need_sync);
  if (st == CUTE_OK && !di.is_auto && grad_b) {
    cute_pair_desc e = *d;
    std::swap(e.cat_a, e.cat_b);
    st = adjoint_pass(ctx, &e, d_G, grad_b, &need_sync);
  }
  if (ctx->timing) cudaEventRecord(ctx->ev1, ctx->stream);
  cudaFreeAsync(d_G, ctx->stream);
  if (st != CUTE_OK) return st;
  if (need_sync) {
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream));
    int err = 0;
    CUDA_OR_FAIL(cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
      CUDA_OR_FAIL(cudaMemset(ctx->d_err, 0, sizeof(int)));
      return fail(ctx, (cute_status)err, "the adjoint kernel reported an error");
    }
  }
  return CUTE_OK;
}

}  // namespace cute

extern "C" {

cute_status cute_count_pairs(cute_ctx *ctx, const cute_pair_desc *d, uint64_t *counts,
                             uint64_t *oor, double *wsum) {
  ENTER(ctx);
  if (!d) return fail(ctx, CUTE_E_INVALID, "descriptor is NULL");
  uint64_t *const cs[1] = {counts};
  double *const ws[1] = {wsum};
  return count_driver(ctx, 1, d, cs, ws, oor);
}

cute_status cute_count_pairs_batched(cute_ctx *ctx, int32_t n, const cute_pair_desc *d,
                                     uint64_t *const *counts, double *const *wsum) {
  ENTER(ctx);
  if (n < 1 || !d || !counts) return fail(ctx, CUTE_E_INVALID, "bad arguments");
  return count_driver(ctx, n, d, counts, wsum, nullptr);
}

cute_status cute_count_pairs_adjoint(cute_ctx *ctx, const cute_pair_desc *d, const double *G,
                                     double *grad_a, double *grad_b) {
  ENTER(ctx);
  return adjoint_driver(ctx, d, G, grad_a, grad_b);
}


cute_status cute_autotune(cute_ctx *ctx, int32_t n, const cute_pair_desc *d, int32_t tune_cells,
                          int64_t max_items, cute_tuning *out) {
  ENTER(ctx);
  if (n < 1 || !d) return fail(ctx, CUTE_E_INVALID, "no descriptors");
  if (max_items <= 0) max_items = (int64_t)1 << 40;
  const int acc = d[0].weighted ? 1 : 0;
  // the geometries the descriptors use, each with every catalog on it (all
  // of them are rebuilt together, so counts between them stay possible)
  std::map<int, std::vector<int32_t>> groups;
  for (int i = 0; i < n; i++) {
    for (int32_t id : {d[i].cat_a, d[i].cat_b}) {
      auto it = ctx->cats.find(id);
      if (it == ctx->cats.end() || it->second.geom < 0)
        return fail(ctx, CUTE_E_STATE, "descriptor catalog missing or without grid");
      groups[it->second.geom];
    }
  }
  for (auto &kv : ctx->cats)
    if (groups.count(kv.second.geom)) groups[kv.second.geom].push_back(kv.first);
  auto rebuild = [&](int k) -> cute_status {
    std::map<int, std::vector<int32_t>> next;
    for (auto &kv : groups) {
      const Geometry g = ctx->geoms[kv.first];
      std::vector<Catalog *> cs;
      for (int32_t id : kv.second) cs.push_back(&ctx->cats[id]);
      CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream));
      ctx->clear_caches();
      cute_status st = grid_build(ctx, cs, g.reach, k);
      if (st != CUTE_OK) return st;
      next[cs[0]->geom] = kv.second;
    }
    groups.swap(next);
    return CUTE_OK;
  };
  const int k0 = ctx->geoms[groups.begin()->first].kreq;
  std::vector<int> ks = tune_cells ? std::vector<int>{2, 3, 4} : std::vector<int>{k0};
  const int save_hp = ctx->hp_override, save_w = ctx->warps_override, save_s = ctx->slice_override;
  cute_tuning best{k0, 0, 0, 0, INFINITY};
  cute_status st = CUTE_OK;
  // small counts (fewer than 1e10 object pairs in all) also try short
  // slices: more, shorter work items per warp balance a launch of a few
  // thousand items (c1: 20k objects, 57 -> 44 us at 64 neighbours)
  double npairs = 0;
  for (int i = 0; i < n; i++)
    npairs += (double)ctx->cats[d[i].cat_a].n * (double)ctx->cats[d[i].cat_b].n;
  const std::vector<int> slices = npairs < 1e10 ? std::vector<int>{64, 256, 1024, 2048, 4096}
                                                : std::vector<int>{1024, 2048, 4096};
  for (int k : ks) {
    if (tune_cells && (st = rebuild(k)) != CUTE_OK) break;
    for (int hp : {2, 4})
      for (int warps : {8, 12, 16, 20})
        for (int slice : slices) {
          ctx->hp_override = hp;
          ctx->warps_override = warps;
          ctx->slice_override = slice;
          Prepared pr;
          if (prepare(ctx, n, d, acc, false, pr) != CUTE_OK) continue;
          if (pr.warps != warps) continue;  // did not fit in shared memory
          const int nb = pr.p.n0 * pr.p.n1;
          const size_t cnt = sizeof(unsigned long long) * (size_t)nb * n;
          const size_t ws = acc ? sizeof(double) * (size_t)nb * n : 0;
          if (ensure_scratch(ctx, cnt + ws + 256) != CUTE_OK) continue;
          pr.p.out_counts = (unsigned long long *)ctx->d_scratch;
          pr.p.out_wsum = acc ? (double *)((char *)ctx->d_scratch + ((cnt + 255) & ~(size_t)255)) : nullptr;
          // an evenly spread sample of the items (they run in home-row order)
          if (pr.p.total > max_items) {
            pr.p.item_stride = (pr.p.total + max_items - 1) / max_items;
            pr.p.total = (pr.p.total + pr.p.item_stride - 1) / pr.p.item_stride;
          }
          if (pr.p.total <= 0) continue;
          float ms = 0;
          for (int rep = 0; rep < 2; rep++) {  // the first run warms up
            CUDA_OR_FAIL(cudaMemsetAsync(ctx->d_ticket, 0, kCounterWords * sizeof(unsigned long long), ctx->stream));
            CUDA_OR_FAIL(cudaEventRecord(ctx->ev0, ctx->stream));
            CUDA_OR_FAIL(launch_prepared(ctx, pr, (int)d[0].kind));
            CUDA_OR_FAIL(cudaEventRecord(ctx->ev1, ctx->stream));
            CUDA_OR_FAIL(cudaEventSynchronize(ctx->ev1));
            CUDA_OR_FAIL(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
          }
          // compare by time per item so shapes with different item sizes
          // are compared on the same work: scale to the full item count
          const double full = (double)ms * ((double)pr.ts->items / (double)pr.p.total);
          if (full < best.ms) best = cute_tuning{k, hp, warps, slice, (float)full};
        }
  }
  ctx->hp_override = save_hp;
  ctx->warps_override = save_w;
  ctx->slice_override = save_s;
  if (st != CUTE_OK) return st;
  if (!std::isfinite(best.ms)) return fail(ctx, CUTE_E_UNSUPPORTED, "no launch shape could run");
  if (tune_cells && best.cells_per_reach != ks.back()) {
    st = rebuild(best.cells_per_reach);
    if (st != CUTE_OK) return st;
  }
  std::vector<DescInfo> dis(n);
  for (int i = 0; i < n; i++) {
    st = validate_desc(ctx, &d[i], dis[i]);
    if (st != CUTE_OK) return st;
    if (!dis[i].is_auto && dis[i].B->n > dis[i].A->n) std::swap(dis[i].A, dis[i].B);
  }
  ctx->tuned[tuning_key(dis, acc, false)] = best;
  if (out) *out = best;
  return CUTE_OK;
}

}  // extern "C"

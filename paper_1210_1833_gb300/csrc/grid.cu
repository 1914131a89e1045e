// grid.cu -- catalog staging and the counting-sort cell grid (Sec. 3.3).
//
// A catalog is kept on the device FP64 in upload order and, once a grid is
// built, cell-sorted as FP32 (x, y, z, w) float4 offsets from the grid
// centre, their FP32 remainders (the re-test's double-float stage) and a
// FP64 SoA copy (the canonical formulas).  The grid is a counting sort: cell
// id and rank within the cell per object (one atomic per object), an
// exclusive scan over cells, and a scatter.  Device blocks come from the
// context's stream-ordered pool.
#include "cute_internal.h"

#include <cfloat>
#include <cstring>

namespace cute {

// ------------------------------------------------------------------ staging stats
// Per-block partial reductions of a catalog: min/max per axis, max |x| per
// axis, min and max |x|^2 (observer at the origin), and the number of
// coordinates outside [0, L) (periodic) or not finite.
struct StageStats {
  double lo[3], hi[3], amax[3], r2min;
  unsigned long long bad;
  double r2max;
};

__global__ void k_stage_stats(const double *__restrict__ xyz, long long n, int periodic, double L,
                              StageStats *__restrict__ out) {
  __shared__ double s_lo[3][256], s_hi[3][256], s_am[3][256], s_r2[256], s_r2x[256];
  __shared__ unsigned long long s_bad[256];
  double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
  double am[3] = {0, 0, 0}, r2m = DBL_MAX, r2x = 0;
  unsigned long long bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double r2 = 0;
    for (int k = 0; k < 3; k++) {
      double x = xyz[3 * i + k];
      if (!(x == x) || x > DBL_MAX || x < -DBL_MAX) bad++;
      if (periodic && !(x >= 0.0 && x < L)) bad++;
      lo[k] = fmin(lo[k], x);
      hi[k] = fmax(hi[k], x);
      am[k] = fmax(am[k], fabs(x));
      r2 += x * x;
    }
    r2m = fmin(r2m, r2);
    r2x = fmax(r2x, r2);
  }
  int t = threadIdx.x;
  for (int k = 0; k < 3; k++) { s_lo[k][t] = lo[k]; s_hi[k][t] = hi[k]; s_am[k][t] = am[k]; }
  s_r2[t] = r2m;
  s_r2x[t] = r2x;
  s_bad[t] = bad;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) {
      for (int k = 0; k < 3; k++) {
        s_lo[k][t] = fmin(s_lo[k][t], s_lo[k][t + s]);
        s_hi[k][t] = fmax(s_hi[k][t], s_hi[k][t + s]);
        s_am[k][t] = fmax(s_am[k][t], s_am[k][t + s]);
      }
      s_r2[t] = fmin(s_r2[t], s_r2[t + s]);
      s_r2x[t] = fmax(s_r2x[t], s_r2x[t + s]);
      s_bad[t] += s_bad[t + s];
    }
    __syncthreads();
  }
  if (t == 0) {
    StageStats st;
    for (int k = 0; k < 3; k++) { st.lo[k] = s_lo[k][0]; st.hi[k] = s_hi[k][0]; st.amax[k] = s_am[k][0]; }
    st.r2min = s_r2[0];
    st.bad = s_bad[0];
    st.r2max = s_r2x[0];
    out[blockIdx.x] = st;
  }
}

// Integer weights: out[0] = the largest weight's bits (non-negative floats
// order like their bits), out[1] = the number of weights that are not
// integers in [0, 2048].
__global__ void k_weight_stats(const float *__restrict__ w, long long n,
                               unsigned *__restrict__ out) {
  unsigned mx = 0, bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = w[i];
    if (!(v >= 0.0f && v <= 2048.0f) || v != rintf(v)) bad++;
    else mx = max(mx, __float_as_uint(v));
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], mx);
    if (bad) atomicAdd(&out[1], bad);
  }
}

// ------------------------------------------------------------------ grid kernels
struct GridDev {
  double lo[3];     // cell origin of the geometry
  double a[3];      // cell sides
  int nc[3];
  double fo[3];     // FP32 frame origin (geometry centre)
};

__device__ __forceinline__ int cell_axis(double x, double lo, double a, int n) {
  double f = floor((x - lo) / a);
  int c = (f < 0.0) ? 0 : (f >= (double)n ? n - 1 : (int)f);
  return c;
}

__global__ void k_cell_assign(const double *__restrict__ xyz, int n, GridDev g,
                              int *__restrict__ cid, int *__restrict__ rank,
                              int *__restrict__ cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cx = cell_axis(xyz[3 * i], g.lo[0], g.a[0], g.nc[0]);
  int cy = cell_axis(xyz[3 * i + 1], g.lo[1], g.a[1], g.nc[1]);
  int cz = cell_axis(xyz[3 * i + 2], g.lo[2], g.a[2], g.nc[2]);
  int c = (cz * g.nc[1] + cy) * g.nc[0] + cx;
  cid[i] = c;
  rank[i] = atomicAdd(&cnt[c], 1);
}

// Exclusive scan of cnt[0..m) into start[0..m], in three passes: the sum of
// every block of kScanBlock cells, an exclusive scan of those sums in one
// block, then each block's own scan offset by its sum's prefix.
constexpr int kScanThreads = 512, kScanPer = 8, kScanBlock = kScanThreads * kScanPer;

// block-wide exclusive scan of one int per thread; returns the block total
__device__ int block_scan_int(int v, int &excl) {
  __shared__ int warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  int off = 0, tot = 0;
  for (int w = 0; w < kScanThreads / 32; w++) {
    if (w < warp) off += warp_tot[w];
    tot += warp_tot[w];
  }
  __syncthreads();
  excl = off + x - v;
  return tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const int *__restrict__ cnt, int m,
                                                            int *__restrict__ bsum) {
  const int base = blockIdx.x * kScanBlock;
  int v = 0;
  for (int k = 0; k < kScanPer; k++) {
    const int i = base + k * kScanThreads + threadIdx.x;
    if (i < m) v += cnt[i];
  }
  int excl;
  const int tot = block_scan_int(v, excl);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(int *__restrict__ bsum, int nblocks,
                                                           int *__restrict__ start, int m) {
  int carry = 0;
  for (int b0 = 0; b0 < nblocks; b0 += kScanThreads) {
    const int b = b0 + threadIdx.x;
    const int v = b < nblocks ? bsum[b] : 0;
    int excl;
    const int tot = block_scan_int(v, excl);
    if (b < nblocks) bsum[b] = carry + excl;
    carry += tot;
  }
  if (threadIdx.x == 0) start[m] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int *__restrict__ cnt, int m,
                                                             const int *__restrict__ bsum,
                                                             int *__restrict__ start) {
  const int base = blockIdx.x * kScanBlock + threadIdx.x * kScanPer;  // consecutive cells
  int v[kScanPer], sum = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; k++) {
    v[k] = base + k < m ? cnt[base + k] : 0;
    sum += v[k];
  }
  int excl;
  block_scan_int(sum, excl);
  int run = bsum[blockIdx.x] + excl;
#pragma unroll
  for (int k = 0; k < kScanPer; k++) {
    if (base + k < m) start[base + k] = run;
    run += v[k];
  }
}

// posq (open grids): the FP32 offsets with q = |x|^2 - q0 (observer
// frame, FP64, rounded once to FP32) in place of the weight, the per-object
// half of the (r, mu) counts' s.l = |x_j|^2 - |x_i|^2.
__global__ void k_scatter(const double *__restrict__ xyz, const float *__restrict__ w, int n,
                          GridDev g, const int *__restrict__ cid, const int *__restrict__ rank,
                          const int *__restrict__ start, float4 *__restrict__ pos,
                          float4 *__restrict__ lo, double *__restrict__ s64,
                          int *__restrict__ perm, float4 *__restrict__ posq, double q0) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int d = start[cid[i]] + rank[i];
  double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  // FP32 frame offsets and their remainders (offset - FP32 offset is exact
  // in FP64; its FP32 rounding leaves pos + lo within 2^-48 of the offset)
  const double ox = x - g.fo[0], oy = y - g.fo[1], oz = z - g.fo[2];
  float4 p;
  p.x = (float)ox;
  p.y = (float)oy;
  p.z = (float)oz;
  p.w = w ? w[i] : 1.0f;
  pos[d] = p;
  lo[d] = make_float4((float)(ox - (double)p.x), (float)(oy - (double)p.y),
                      (float)(oz - (double)p.z), 0.0f);
  s64[d] = x;
  s64[(size_t)n + d] = y;
  s64[2 * (size_t)n + d] = z;
  perm[d] = i;
  if (posq) {
    const double q = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)), q0);
    posq[d] = make_float4(p.x, p.y, p.z, (float)q);
  }
}

// cells holding at least one object (grid-stride, one atomic per warp)
__global__ void k_occupied(const int *__restrict__ cnt, long long ncell, int *__restrict__ out) {
  int c = 0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < ncell;
       q += (long long)gridDim.x * blockDim.x)
    c += cnt[q] > 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// ------------------------------------------------------------------ host side
static cute_status fail(cute_ctx *ctx, cute_status st, const std::string &m) {
  ctx->err = m;
  return st;
}

#define CUDA_OR_FAIL(call)                                                         \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? CUTE_E_OOM : CUTE_E_CUDA, \
                  std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

cute_status ensure_scratch(cute_ctx *ctx, size_t bytes) {
  if (ctx->scratch_bytes >= bytes) return CUTE_OK;
  if (ctx->d_scratch) {
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->d_scratch);
    ctx->d_scratch = nullptr;
    ctx->scratch_bytes = 0;
  }
  size_t want = bytes + bytes / 4;
  CUDA_OR_FAIL(cudaMalloc(&ctx->d_scratch, want));
  ctx->scratch_bytes = want;
  return CUTE_OK;
}

cute_status catalog_stage(cute_ctx *ctx, Catalog &c, const double *xyz, const float *w) {
  const long long n = c.n;
  if (n > 0) {
    CUDA_OR_FAIL(dev_alloc(ctx, (void **)&c.d_xyz, sizeof(double) * 3 * (size_t)n));
    CUDA_OR_FAIL(cudaMemcpyAsync(c.d_xyz, xyz, sizeof(double) * 3 * (size_t)n, cudaMemcpyDefault,
                                 ctx->stream));
    if (w) {
      CUDA_OR_FAIL(dev_alloc(ctx, (void **)&c.d_w, sizeof(float) * (size_t)n));
      CUDA_OR_FAIL(cudaMemcpyAsync(c.d_w, w, sizeof(float) * (size_t)n, cudaMemcpyDefault,
                                   ctx->stream));
    }
  }
  // statistics and validation
  int blocks = 1;
  if (n > 0) blocks = (int)std::min<long long>((n + 255) / 256, 4LL * ctx->sm_count);
  cute_status st = ensure_scratch(ctx, sizeof(StageStats) * blocks);
  if (st != CUTE_OK) return st;
  std::vector<StageStats> part(blocks);
  if (n > 0) {
    k_stage_stats<<<blocks, 256, 0, ctx->stream>>>(c.d_xyz, n, c.boundary == CUTE_PERIODIC, c.L,
                                                   (StageStats *)ctx->d_scratch);
    CUDA_OR_FAIL(cudaGetLastError());
    CUDA_OR_FAIL(cudaMemcpyAsync(part.data(), ctx->d_scratch, sizeof(StageStats) * blocks,
                                 cudaMemcpyDeviceToHost, ctx->stream));
  }
  CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream));
  unsigned long long bad = 0;
  double r2min = DBL_MAX, r2max = 0;
  for (int k = 0; k < 3; k++) { c.lo[k] = DBL_MAX; c.hi[k] = -DBL_MAX; c.absmax[k] = 0; }
  if (n > 0) {
    for (auto &p : part) {
      for (int k = 0; k < 3; k++) {
        c.lo[k] = std::min(c.lo[k], p.lo[k]);
        c.hi[k] = std::max(c.hi[k], p.hi[k]);
        c.absmax[k] = std::max(c.absmax[k], p.amax[k]);
      }
      r2min = std::min(r2min, p.r2min);
      r2max = std::max(r2max, p.r2max);
      bad += p.bad;
    }
  } else {
    for (int k = 0; k < 3; k++) { c.lo[k] = 0; c.hi[k] = 0; }
    r2min = 0;
  }
  c.rmin = std::sqrt(r2min);
  c.rmax = std::sqrt(r2max);
  c.wint = -1;
  if (w && n > 0) {
    st = ensure_scratch(ctx, 2 * sizeof(unsigned));
    if (st != CUTE_OK) return st;
    unsigned h[2] = {0, 0};
    CUDA_OR_FAIL(cudaMemsetAsync(ctx->d_scratch, 0, 2 * sizeof(unsigned), ctx->stream));
    k_weight_stats<<<blocks, 256, 0, ctx->stream>>>(c.d_w, n, (unsigned *)ctx->d_scratch);
    CUDA_OR_FAIL(cudaGetLastError());
    CUDA_OR_FAIL(cudaMemcpyAsync(h, ctx->d_scratch, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream));
    float mx;
    std::memcpy(&mx, &h[0], 4);
    if (h[1] == 0) c.wint = (int)mx;
  }
  if (bad) {
    return fail(ctx, CUTE_E_INVALID,
                c.boundary == CUTE_PERIODIC
                    ? "catalog has coordinates outside [0, box_L) or not finite"
                    : "catalog has coordinates that are not finite");
  }
  return CUTE_OK;
}

static void free_grid(cute_ctx *ctx, Catalog &c) {
  dev_free(ctx, c.d_pos); c.d_pos = nullptr;
  dev_free(ctx, c.d_posq); c.d_posq = nullptr;
  dev_free(ctx, c.d_lo); c.d_lo = nullptr;
  dev_free(ctx, c.d_s64); c.d_s64 = nullptr;
  dev_free(ctx, c.d_perm); c.d_perm = nullptr;
  dev_free(ctx, c.d_cell_start); c.d_cell_start = nullptr;
  pinned_put(ctx, c.h_cell_start, c.h_cap);
  c.h_cell_start = nullptr;
  c.h_cap = 0;
  c.chunk_cache.clear();
  c.geom = -1;
}

void catalog_release(cute_ctx *ctx, Catalog &c) {
  free_grid(ctx, c);
  dev_free(ctx, c.d_xyz); c.d_xyz = nullptr;
  dev_free(ctx, c.d_w); c.d_w = nullptr;
}

cute_status grid_build(cute_ctx *ctx, const std::vector<Catalog *> &cats, const double reach[3],
                       int kreq) {
  const Catalog &c0 = *cats[0];
  Geometry g;
  g.periodic = (c0.boundary == CUTE_PERIODIC);
  g.L = c0.L;
  for (int k = 0; k < 3; k++) g.reach[k] = reach[k];
  double lo[3], hi[3];
  for (int k = 0; k < 3; k++) {
    lo[k] = DBL_MAX; hi[k] = -DBL_MAX; g.absmax[k] = 0;
  }
  g.rmin = DBL_MAX;
  g.rmax = 0;
  bool any = false;
  for (Catalog *c : cats) {
    if (c->n == 0) continue;
    any = true;
    for (int k = 0; k < 3; k++) {
      lo[k] = std::min(lo[k], c->lo[k]);
      hi[k] = std::max(hi[k], c->hi[k]);
      g.absmax[k] = std::max(g.absmax[k], c->absmax[k]);
    }
    g.rmin = std::min(g.rmin, c->rmin);
    g.rmax = std::max(g.rmax, c->rmax);
  }
  if (!any) {
    for (int k = 0; k < 3; k++) { lo[k] = 0; hi[k] = 1; }
    g.rmin = 0;
  }
  // (r, mu): q = |x|^2 - q0 with q0 in the middle of the catalogs' range of
  // |x|^2, so |q| <= qd; qd also covers the FP64 evaluation of |x|^2 - q0
  // (four roundings of values up to rmax^2)
  g.q0 = 0.5 * (g.rmin * g.rmin + g.rmax * g.rmax);
  g.qd = 0.5 * (g.rmax * g.rmax - g.rmin * g.rmin) * (1.0 + 1e-12) + 1e-15 * g.rmax * g.rmax;
  for (int k = 0; k < 3; k++) {
    // cells no smaller than reach/k (with a relative margin that absorbs the
    // rounding of the cell assignment), so objects more than k cells apart
    // on an axis are farther apart than the reach on that axis.  Rows of
    // cells run along x and a neighbour row is a contiguous range of objects
    // whatever its length, so x is cut kXFine times finer: the ends of each
    // row range then follow the reach closely at no cost in work items.
    const int kx_req = (k == 0) ? kreq * kXFine : kreq;
    const long long ncap = (k == 0) ? 8192 : 1024;
    double amin = reach[k] * (1.0 + 1e-9) / kx_req + 1e-300;
    int kk = kx_req;
    if (g.periodic) {
      double L = g.L;
      long long n = (long long)std::floor(L / amin);
      // the (2k+1)-cell stencil must not wrap onto itself: raise k if needed
      while (n < 2 * kk + 1 && kk < 16 * kx_req) {
        kk++;
        amin = reach[k] * (1.0 + 1e-9) / kk + 1e-300;
        n = (long long)std::floor(L / amin);
      }
      if (n < 2 * kk + 1)
        return fail(ctx, CUTE_E_UNSUPPORTED, "periodic reach too large for the box (needs reach <= 0.47 L)");
      n = std::min<long long>(n, ncap);
      g.nc[k] = (int)n;
      g.a[k] = L / (double)n;
      // a stencil of kk cells must still cover the reach after capping n
      kk = (int)std::ceil(reach[k] * (1.0 + 1e-9) / g.a[k]);
      if (kk < 1) kk = 1;
      if (2 * kk + 1 > g.nc[k])
        return fail(ctx, CUTE_E_UNSUPPORTED, "periodic reach too large for the box (needs reach <= 0.47 L)");
      g.k[k] = kk;
      g.origin[k] = 0.0;
      g.xmax[k] = 0.5 * L;   // FP32 frame centred on the box
    } else {
      double ext = hi[k] - lo[k];
      long long n = (long long)std::floor(ext / amin) + 1;
      n = std::max<long long>(1, std::min<long long>(n, ncap));
      double a = std::max(amin, ext / (double)n * (1.0 + 1e-12));
      g.nc[k] = (int)n;
      g.a[k] = a;
      g.k[k] = (int)std::max<double>(1.0, std::ceil(reach[k] * (1.0 + 1e-9) / a));
      g.origin[k] = lo[k];
      g.xmax[k] = 0.5 * ext * (1.0 + 1e-12) + 1e-300;
    }
  }
  long long ncell = (long long)g.nc[0] * g.nc[1] * g.nc[2];
  if (ncell > (1LL << 28)) return fail(ctx, CUTE_E_UNSUPPORTED, "too many cells");
  // the counting kernels' padding sentinels sit at 1e9 in the FP32 grid
  // frame (offsets from the grid centre): real objects must stay within 1e8
  for (int k = 0; k < 3; k++)
    if (!(g.xmax[k] <= 1e8))
      return fail(ctx, CUTE_E_UNSUPPORTED, "catalog extent beyond 2e8 on an axis");
  g.id = ctx->next_geom++;
  g.version = ++ctx->version_counter;
  g.kreq = kreq;

  GridDev gd;
  for (int k = 0; k < 3; k++) {
    gd.lo[k] = g.origin[k];
    gd.a[k] = g.a[k];
    gd.nc[k] = g.nc[k];
    gd.fo[k] = g.periodic ? 0.5 * g.L : 0.5 * (lo[k] + hi[k]);
    if (!any) gd.fo[k] = 0;
    g.fo[k] = gd.fo[k];
  }
  // the FP32 frame spans at most xmax from its centre on each axis
  for (Catalog *c : cats) {
    free_grid(ctx, *c);
    const int n = (int)c->n;
    CUDA_OR_FAIL(dev_alloc(ctx, (void **)&c->d_cell_start, sizeof(int) * (size_t)(ncell + 1)));
    if (n > 0) {
      CUDA_OR_FAIL(dev_alloc(ctx, (void **)&c->d_pos, sizeof(float4) * (size_t)n));
      if (!g.periodic) CUDA_OR_FAIL(dev_alloc(ctx, (void **)&c->d_posq, sizeof(float4) * (size_t)n));
      CUDA_OR_FAIL(dev_alloc(ctx, (void **)&c->d_lo, sizeof(float4) * (size_t)n));
      CUDA_OR_FAIL(dev_alloc(ctx, (void **)&c->d_s64, sizeof(double) * 3 * (size_t)n));
      CUDA_OR_FAIL(dev_alloc(ctx, (void **)&c->d_perm, sizeof(int) * (size_t)n));
    }
    const int nsb = (int)((ncell + kScanBlock - 1) / kScanBlock);
    size_t need = sizeof(int) * ((size_t)2 * n + (size_t)ncell + (size_t)nsb + 1) + 256;
    cute_status st = ensure_scratch(ctx, need);
    if (st != CUTE_OK) return st;
    int *cid = (int *)ctx->d_scratch;
    int *rank = cid + n;
    int *cnt = rank + n;
    int *bsum = cnt + ncell;
    CUDA_OR_FAIL(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)ncell, ctx->stream));
    if (n > 0) {
      k_cell_assign<<<(n + 255) / 256, 256, 0, ctx->stream>>>(c->d_xyz, n, gd, cid, rank, cnt);
      CUDA_OR_FAIL(cudaGetLastError());
    }
    k_scan_sums<<<nsb, kScanThreads, 0, ctx->stream>>>(cnt, (int)ncell, bsum);
    k_scan_top<<<1, kScanThreads, 0, ctx->stream>>>(bsum, nsb, c->d_cell_start, (int)ncell);
    k_scan_apply<<<nsb, kScanThreads, 0, ctx->stream>>>(cnt, (int)ncell, bsum, c->d_cell_start);
    CUDA_OR_FAIL(cudaGetLastError());
    if (n > 0) {
      k_scatter<<<(n + 255) / 256, 256, 0, ctx->stream>>>(c->d_xyz, c->d_w, n, gd, cid, rank,
                                                          c->d_cell_start, c->d_pos, c->d_lo,
                                                          c->d_s64, c->d_perm, c->d_posq, g.q0);
      CUDA_OR_FAIL(cudaGetLastError());
    }
    // host copy of cell_start and the occupied-cell count (after it), into
    // a pinned block: every catalog's copies are in flight before one sync
    int *occ = bsum + nsb;
    CUDA_OR_FAIL(cudaMemsetAsync(occ, 0, sizeof(int), ctx->stream));
    k_occupied<<<std::min<long long>((ncell + 255) / 256, 4LL * ctx->sm_count), 256, 0,
                 ctx->stream>>>(cnt, ncell, occ);
    CUDA_OR_FAIL(cudaGetLastError());
    CUDA_OR_FAIL(pinned_get(ctx, (size_t)ncell + 2, &c->h_cell_start, &c->h_cap));
    CUDA_OR_FAIL(cudaMemcpyAsync(c->h_cell_start, c->d_cell_start,
                                 sizeof(int) * (size_t)(ncell + 1), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    CUDA_OR_FAIL(cudaMemcpyAsync(c->h_cell_start + ncell + 1, occ, sizeof(int),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    c->geom = g.id;
    c->grid_version = g.version;
  }
  CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream));
  for (Catalog *c : cats) c->occupied_cells = c->h_cell_start[ncell + 1];
  ctx->geoms[g.id] = g;
  return CUTE_OK;
}

}  // namespace cute

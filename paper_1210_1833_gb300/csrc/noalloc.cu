// noalloc.cu -- a counting entry point that allocates no device memory.
//
// cute_count_pairs keeps its per-request device data (binning tables, work
// lists, work counters) in buffers it allocates and caches.  Some callers
// cannot let a library allocate at the moment they count: a framework whose
// caching allocator owns all device memory (a stray cudaMalloc fragments its
// pool or fails once the pool has taken the device), or loops where
// cudaMalloc/cudaFree would synchronise the whole device.
// cute_count_pairs_noalloc serves them: the same counting kernel, with its
// scratch in one fixed file-scope device array that every call on a device
// shares.  The caller passes the outputs (device memory of the context's
// device); the catalogs and their grids are set up beforehand.  Each call
// builds its work-item records on the host (time grows with the number of
// items) and copies them, with the tables, from pageable host memory, a copy
// that waits for the context's stream.
#include "cute_internal.h"
#include "count_kernel.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

namespace cute {
size_t hist_budget(const cute_pair_desc *d, int acc, int hp);  // api.cu
cudaError_t launch_count_mono(const KParams &p, bool periodic, int acc, int hp, int blocks,
                              int threads, size_t smem, cudaStream_t st);
cudaError_t launch_count_sigpi(const KParams &p, bool periodic, int acc, int hp, int blocks,
                               int threads, size_t smem, cudaStream_t st);
cudaError_t launch_count_rmu(const KParams &p, int acc, int hp, int blocks, int threads,
                             size_t smem, cudaStream_t st);
}  // namespace cute

using namespace cute;

// The scratch: 8 MiB on every device that loads the library, held until the
// process exits.  Host code must not use this name as an address (it is a
// host-side stand-in): the device address comes from cudaGetSymbolAddress.
static constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[256];  // device address of the scratch, per device

static cute_status na_fail(cute_ctx *ctx, cute_status st, const std::string &m) {
  ctx->err = m;
  return st;
}

#define NA_CUDA(call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return na_fail(ctx, CUTE_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// device memory of `device` (or managed memory, which every device reaches)
static bool na_is_device(const void *p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == device;
}

static size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" cute_status cute_count_pairs_noalloc(cute_ctx *ctx, const cute_pair_desc *d,
                                                uint64_t *counts, double *wsum) {
  if (!ctx) return CUTE_E_INVALID;
  ctx->err.clear();
  NA_CUDA(cudaSetDevice(ctx->device));
  if (!d || !counts) return na_fail(ctx, CUTE_E_INVALID, "descriptor and counts are required");
  if (!na_is_device(counts, ctx->device) ||
      (d->weighted && (!wsum || !na_is_device(wsum, ctx->device))))
    return na_fail(ctx, CUTE_E_INVALID, "outputs must be device memory of the context's device");
  if (ctx->device < 0 || ctx->device >= 256) return na_fail(ctx, CUTE_E_INVALID, "device index");

  // set-up, once per device, with that device current
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[ctx->device]) {
      void *a = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
      if (e != cudaSuccess || !a)
        return na_fail(ctx, CUTE_E_CUDA,
                       std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      g_noalloc_addr[ctx->device] = a;
    }
    base = g_noalloc_addr[ctx->device];
  }

  DescInfo di;
  cute_status st = validate_desc(ctx, d, di);
  if (st != CUTE_OK) return st;
  if (!di.is_auto && di.B->n > di.A->n) std::swap(di.A, di.B);  // fuller home cells
  const int kind = (int)d->kind;
  const bool two_d = (kind == CUTE_R_MU || kind == CUTE_SIGMA_PI);
  const int acc = d->weighted ? 1 : 0;
  std::vector<DescInfo> dis(1, di);
  ErrorParams ep = error_params(dis, decision_reach(d));

  int hp = ctx->hp_override;
  if (!hp) hp = row_density(*di.A, *di.g) < 2000.0 ? 2 : 4;
  if (!ctx->hp_override && acc == 0 && (kind == CUTE_MONO || kind == CUTE_THETA)) hp = 2;
  const int slice = ctx->slice_override ? ctx->slice_override : 2048;

  // binning plan, chunks and stencil on the host
  Plan P;
  std::string m = plan_build(kind, d->edges0, d->n0, d->edges1, two_d ? d->n1 : 1, ep, 8192,
                             hist_budget(d, acc, hp), !ctx->table_binning, P);
  if (!m.empty()) return na_fail(ctx, CUTE_E_UNSUPPORTED, m);
  std::vector<int4> chunks, stencil;
  if (di.A->n > 0 && di.B->n > 0) {
    const int shape = (kind == CUTE_SIGMA_PI) ? kShapeDiskSlab : kShapeBall;
    chunks_build(*di.g, di.A->h_cell_start, 32 * hp, chunks);
    stencil_build(*di.g, di.is_auto, false, shape, di.need, stencil);
  }
  PairDev pd = pair_dev(di, 0);
  PairWork pw;
  std::memset(&pw, 0, sizeof(pw));
  pw.nchunks = (int32_t)chunks.size();
  pw.nstencil = (int32_t)stencil.size();
  pw.nx = di.g->nc[0];
  pw.ny = di.g->nc[1];
  pw.nz = di.g->nc[2];
  pw.mode = di.is_auto ? kModeAutoHalf : kModeCross;
  pw.periodic = di.g->periodic;
  // the item records, on the host (the same segments as the GPU builder)
  std::vector<int4> items;
  const int32_t *csh = di.B->h_cell_start;
  for (const int4 &c : chunks)
    for (const int4 &r : stencil) {
      Seg sg[3];
      const int ns = entry_segments(pw, csh, c, r, sg);
      for (int k = 0; k < ns; k++)
        for (int js = sg[k].j0; js < sg[k].j1; js += slice)
          items.push_back(item_record(c.x, c.y, sg[k], js, std::min(js + slice, sg[k].j1), 0));
    }

  // scratch layout: counters | pair | double-float pair | item records |
  // tables | bands | edges (FP64, then hi + lo)
  const size_t o_cnt = 0;
  const size_t o_pair = na_align(o_cnt + kCounterWords * sizeof(unsigned long long));
  const size_t o_pdf = na_align(o_pair + sizeof(PairDev));
  const size_t o_items = na_align(o_pdf + sizeof(PairDF));
  const size_t o_lut = na_align(o_items + items.size() * sizeof(int4));
  const size_t o_band = na_align(o_lut + P.lut.size() * sizeof(uint32_t));
  const size_t o_e0 = na_align(o_band + P.band.size() * sizeof(float));
  const size_t o_e1 = na_align(o_e0 + P.E0.size() * sizeof(double));
  const size_t o_e0df = na_align(o_e1 + P.E1.size() * sizeof(double));
  const size_t o_e1df = na_align(o_e0df + P.E0df.size() * sizeof(float));
  const size_t total = na_align(o_e1df + P.E1df.size() * sizeof(float));
  if (total > kNoAllocScratchBytes)
    return na_fail(ctx, CUTE_E_INVALID,
                   "request needs " + std::to_string(total) +
                       " bytes of scratch; cute_count_pairs_noalloc has 8 MiB (use fewer work "
                       "items: smaller catalogs, or cute_count_pairs)");
  unsigned char *dev = (unsigned char *)base;
  pd.df = (const PairDF *)(dev + o_pdf);
  const PairDF pdf = pair_df(di);
  std::vector<unsigned char> img(total, 0);  // counters start at zero
  std::memcpy(img.data() + o_pair, &pd, sizeof(PairDev));
  std::memcpy(img.data() + o_pdf, &pdf, sizeof(PairDF));
  std::memcpy(img.data() + o_items, items.data(), items.size() * sizeof(int4));
  std::memcpy(img.data() + o_lut, P.lut.data(), P.lut.size() * sizeof(uint32_t));
  std::memcpy(img.data() + o_band, P.band.data(), P.band.size() * sizeof(float));
  std::memcpy(img.data() + o_e0, P.E0.data(), P.E0.size() * sizeof(double));
  std::memcpy(img.data() + o_e1, P.E1.data(), P.E1.size() * sizeof(double));
  std::memcpy(img.data() + o_e0df, P.E0df.data(), P.E0df.size() * sizeof(float));
  std::memcpy(img.data() + o_e1df, P.E1df.data(), P.E1df.size() * sizeof(float));
  NA_CUDA(cudaMemcpyAsync(dev, img.data(), total, cudaMemcpyHostToDevice, ctx->stream));

  const int nb = P.n0 * P.n1;
  NA_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint64_t) * nb, ctx->stream));
  if (acc == 1) NA_CUDA(cudaMemsetAsync(wsum, 0, sizeof(double) * nb, ctx->stream));

  KParams p;
  std::memset(&p, 0, sizeof(p));
  p.items = (const int4 *)(dev + o_items);
  p.total = (long long)items.size();
  p.item_stride = 1;
  p.pairs = (const PairDev *)(dev + o_pair);
  p.lut = (const uint32_t *)(dev + o_lut);
  p.lut_words = (int)P.lut.size();
  p.ax[0] = P.ax[0];
  p.ax[1] = P.ax[1];
  p.band = (const float2 *)(dev + o_band);
  p.band_words = (int)P.band.size() / 2;
  p.mu_eps_base = P.mu_eps_base;
  p.far = P.far;
  cull_params(std::vector<DescInfo>{di}, d, 1, p);
  p.E0 = (const double *)(dev + o_e0);
  p.E1 = (const double *)(dev + o_e1);
  p.E0df = (const float2 *)(dev + o_e0df);
  p.E1df = (const float2 *)(dev + o_e1df);
  p.n0 = P.n0;
  p.n1 = P.n1;
  p.slots1 = P.slots1;
  p.nslots = P.nslots;
  p.R = P.R;
  p.slice = slice;
  p.out_counts = (unsigned long long *)counts;
  p.out_wsum = acc == 1 ? wsum : nullptr;
  p.ticket = (unsigned long long *)(dev + o_cnt);
  p.stats = (unsigned long long *)(dev + o_cnt) + 1;
  p.err = ctx->d_err;

  SmemLayout L = smem_layout(p.lut_words, p.band_words, P.nslots, P.R, hp, acc,
                             kind == CUTE_R_MU && acc != 0, kind == CUTE_R_MU || acc != 0);
  const int wmax = count_max_warps(kind == CUTE_MONO || kind == CUTE_THETA, hp, acc);
  int warps = ctx->warps_override ? std::min(ctx->warps_override, wmax) : wmax;
  while (warps > 1 && (size_t)L.lut_bytes + (size_t)warps * L.warp_bytes > ctx->smem_optin) warps--;
  const size_t smem = (size_t)L.lut_bytes + (size_t)warps * L.warp_bytes;
  if (smem > ctx->smem_optin)
    return na_fail(ctx, CUTE_E_UNSUPPORTED, "binning tables do not fit in shared memory");
  if (p.total == 0) return CUTE_OK;
  const bool per = di.g->periodic;
  const int threads = warps * 32, blocks = ctx->sm_count;
  cudaError_t e;
  switch (kind) {
    case CUTE_MONO: e = launch_count_mono(p, per, acc, hp, blocks, threads, smem, ctx->stream); break;
    case CUTE_THETA: e = launch_count_mono(p, false, acc, hp, blocks, threads, smem, ctx->stream); break;
    case CUTE_SIGMA_PI: e = launch_count_sigpi(p, per, acc, hp, blocks, threads, smem, ctx->stream); break;
    default: e = launch_count_rmu(p, acc, hp, blocks, threads, smem, ctx->stream); break;
  }
  if (e != cudaSuccess) return na_fail(ctx, CUTE_E_CUDA, cudaGetErrorString(e));
  return CUTE_OK;
}

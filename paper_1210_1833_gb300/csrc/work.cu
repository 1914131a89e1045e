// work.cu -- the work decomposition of a count, on the GPU.
//
// A count's work entries are (home chunk, stencil row) of each pair set; an
// entry meets up to three contiguous segments of catalog B (entry_segments)
// and splits into one work item per `slice` neighbours of each segment.
// Three kernels turn the entries into item prefix sums (item counts per
// entry with per-block sums, an exclusive scan of the block sums in one
// block, the block-local scans); a fourth writes every entry's item records
// at its prefix, the list the counting kernel's ticket walks.  Nothing here
// depends on the host beyond the chunk and stencil lists.
#include "cute_internal.h"
#include "count_kernel.cuh"
#include "work_pairs.h"

#include <algorithm>

namespace cute {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;                        // entries per thread
constexpr int kScanBlock = kScanThreads * kScanPer;  // entries per block

// Items of entry e, and the pairs its segments present to the counting
// kernel: every (home, neighbour) pair, j > i on the home run's own cells
// (kSegSelf), without i = j on a full stencil's home row (kSegNoSelfPair).
__device__ __forceinline__ int entry_items(const PairWork *__restrict__ pairs,
                                           const int *__restrict__ ebase, int npairs, int e,
                                           int slice, unsigned long long &npair) {
  const int pi = pair_of_entry(ebase, npairs, e);
  const PairWork &pd = pairs[pi];
  const int local = e - ebase[pi];
  const int ci = local / pd.nstencil, ri = local - ci * pd.nstencil;
  const int4 c = pd.chunks[ci];
  Seg s[3];
  const int ns = entry_segments(pd, pd.csB, c, pd.stencil[ri], s);
  int items = 0;
  for (int k = 0; k < ns; k++) {
    items += (s[k].j1 - s[k].j0 + slice - 1) / slice;
    npair += segment_pairs(c, s[k]);
  }
  return items;
}

// block-wide exclusive scan of one value per thread; returns the block total
__device__ long long block_scan(long long v, long long &excl) {
  __shared__ long long warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  long long off = 0, tot = 0;
  for (int w = 0; w < kScanThreads / 32; w++) {
    if (w < warp) off += warp_tot[w];
    tot += warp_tot[w];
  }
  __syncthreads();
  excl = off + x - v;
  return tot;
}

__global__ void __launch_bounds__(kScanThreads) k_entry_counts(
    const PairWork *__restrict__ pairs, const int *__restrict__ ebase, int npairs, int nentries,
    int slice, int *__restrict__ cnt, long long *__restrict__ bsum,
    unsigned long long *__restrict__ spairs) {
  const int base = blockIdx.x * kScanBlock;
  long long sum = 0;
  unsigned long long np = 0;
  for (int k = 0; k < kScanPer; k++) {
    const int e = base + k * kScanThreads + threadIdx.x;  // coalesced stores
    if (e < nentries) {
      const int c = entry_items(pairs, ebase, npairs, e, slice, np);
      cnt[e] = c;
      sum += c;
    }
  }
  long long excl;
  const long long tot = block_scan(sum, excl);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
  for (int o = 16; o > 0; o >>= 1) np += __shfl_xor_sync(kFull, np, o);
  if ((threadIdx.x & 31) == 0 && np) atomicAdd(spairs, np);
}

// exclusive scan of the block sums, in place, by one block
__global__ void __launch_bounds__(kScanThreads) k_scan_bsums(long long *__restrict__ bsum,
                                                             int nblocks) {
  long long carry = 0;
  for (int b0 = 0; b0 < nblocks; b0 += kScanThreads) {
    const int b = b0 + threadIdx.x;
    const long long v = b < nblocks ? bsum[b] : 0;
    long long excl;
    const long long tot = block_scan(v, excl);
    if (b < nblocks) bsum[b] = carry + excl;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_entries(
    const int *__restrict__ cnt, const long long *__restrict__ bsum, int nentries, int nblocks,
    long long *__restrict__ eprefix) {
  // thread t scans its kScanPer consecutive entries
  const int base = blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
  int v[kScanPer];
  long long sum = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; k++) {
    const int e = base + k;
    v[k] = e < nentries ? cnt[e] : 0;
    sum += v[k];
  }
  long long excl;
  const long long tot = block_scan(sum, excl);
  long long run = bsum[blockIdx.x] + excl;
#pragma unroll
  for (int k = 0; k < kScanPer; k++) {
    const int e = base + k;
    if (e < nentries) eprefix[e] = run;
    run += v[k];
  }
  if (blockIdx.x == nblocks - 1 && threadIdx.x == 0) eprefix[nentries] = bsum[blockIdx.x] + tot;
}

__global__ void __launch_bounds__(kScanThreads) k_entry_write(
    const PairWork *__restrict__ pairs, const int *__restrict__ ebase, int npairs, int nentries,
    int slice, const long long *__restrict__ eprefix, int4 *__restrict__ items) {
  const int e = blockIdx.x * kScanThreads + threadIdx.x;
  if (e >= nentries) return;
  const int pi = pair_of_entry(ebase, npairs, e);
  const PairWork &pd = pairs[pi];
  const int local = e - ebase[pi];
  const int ci = local / pd.nstencil, ri = local - ci * pd.nstencil;
  const int4 c = pd.chunks[ci];
  Seg s[3];
  const int ns = entry_segments(pd, pd.csB, c, pd.stencil[ri], s);
  long long o = eprefix[e];
  for (int k = 0; k < ns; k++)
    for (int js = s[k].j0; js < s[k].j1; js += slice)
      items[o++] = item_record(c.x, c.y, s[k], js, min(js + slice, s[k].j1), pi);
}

}  // namespace

int work_bsum_words(int nentries) { return std::max(1, (nentries + kScanBlock - 1) / kScanBlock); }

cudaError_t work_count(const PairWork *d_pairs, const int *d_ebase, int npairs, int nentries,
                       int slice, int *d_cnt, long long *d_bsum, long long *d_eprefix,
                       unsigned long long *d_spairs, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(d_spairs, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (nentries <= 0) return cudaMemsetAsync(d_eprefix, 0, sizeof(long long), st);
  const int nblocks = work_bsum_words(nentries);
  k_entry_counts<<<nblocks, kScanThreads, 0, st>>>(d_pairs, d_ebase, npairs, nentries, slice,
                                                   d_cnt, d_bsum, d_spairs);
  k_scan_bsums<<<1, kScanThreads, 0, st>>>(d_bsum, nblocks);
  k_scan_entries<<<nblocks, kScanThreads, 0, st>>>(d_cnt, d_bsum, nentries, nblocks, d_eprefix);
  return cudaGetLastError();
}

cudaError_t work_write(const PairWork *d_pairs, const int *d_ebase, int npairs, int nentries,
                       int slice, const long long *d_eprefix, int4 *d_items, cudaStream_t st) {
  if (nentries <= 0) return cudaSuccess;
  k_entry_write<<<(nentries + kScanThreads - 1) / kScanThreads, kScanThreads, 0, st>>>(
      d_pairs, d_ebase, npairs, nentries, slice, d_eprefix, d_items);
  return cudaGetLastError();
}

}  // namespace cute

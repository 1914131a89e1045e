// density.cu -- the density-grid estimate of the monopole in a periodic box
// (Sec. 3.4.4).
//
// The catalog is interpolated to an n^3 grid with the triangular-shaped-
// cloud (TSC) kernel, the overdensity delta = rho / mean(rho) - 1 is formed
// at every grid point, and xi(r) is the mean of delta_i delta_j over the
// pairs of distinct grid points whose separation falls in each bin.  On a
// regular periodic grid the pairs at a lag vector d all share one
// separation, so the work is the lag correlation
//     C(d) = sum_i delta_i delta_{i + d}
// for every lag of the half ball |d| a < r_max (each unordered pair once),
// and xi_b = sum_{d in b} C(d) / (n^3 * #lags in b).
//
// Kernels:
//   k_tsc       27 FP64 atomic adds per object into the grid;
//   k_delta     rho -> FP32 delta;
//   k_lagcorr   one CTA per (dy, dz) lag column, lag window and z slab: the
//               rows delta[:, y, z] and delta[:, y + dy, z + dz] (plus the dx
//               halo) are staged in skewed shared memory by cp.async, two
//               stages in flight; each lane sums 16 consecutive dx lags over
//               its blocks of 16 consecutive x (register blocks of 16 x 16);
//               FP32 partial sums over 8 rows are folded into float-float
//               accumulators, so a lag sum carries about the FP32 rounding of
//               those partials.
#include "cute_internal.h"
#include "count_kernel.cuh"  // cp.async helpers

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace cute {

namespace {

constexpr int kMaxGrid = 1024;

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// TSC weights of a particle at grid coordinate u (grid points at integers):
// nearest point i0 = rint(u), d = u - i0 in [-1/2, 1/2]:
// w(i0 - 1) = (1/2 - d)^2 / 2, w(i0) = 3/4 - d^2, w(i0 + 1) = (1/2 + d)^2 / 2
__device__ __forceinline__ void tsc1(double u, int n, int idx[3], double w[3]) {
  const double i0 = rint(u);
  const double d = u - i0;
  const int c = (int)i0;
  idx[0] = wrapi(c - 1, n);
  idx[1] = wrapi(c >= n ? c - n : c, n);
  idx[2] = wrapi(c + 1 >= n ? c + 1 - n : c + 1, n);
  w[0] = 0.5 * (0.5 - d) * (0.5 - d);
  w[1] = 0.75 - d * d;
  w[2] = 0.5 * (0.5 + d) * (0.5 + d);
}

__global__ void k_tsc(const double *__restrict__ xyz, const float *__restrict__ wt, long long np,
                      int n, double inv_a, double *__restrict__ rho, int *__restrict__ bad,
                      double box) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  int ix[3], iy[3], iz[3];
  double wx[3], wy[3], wz[3];
  const double x = xyz[3 * p], y = xyz[3 * p + 1], z = xyz[3 * p + 2];
  if (!(x >= 0.0 && x < box && y >= 0.0 && y < box && z >= 0.0 && z < box)) {
    atomicExch(bad, 1);
    return;
  }
  tsc1(x * inv_a, n, ix, wx);
  tsc1(y * inv_a, n, iy, wy);
  tsc1(z * inv_a, n, iz, wz);
  const double m = wt ? (double)wt[p] : 1.0;
  for (int c = 0; c < 3; c++)
    for (int b = 0; b < 3; b++) {
      const double wzy = m * wz[c] * wy[b];
      const long long row = ((long long)iz[c] * n + iy[b]) * n;
      for (int a = 0; a < 3; a++) atomicAdd(&rho[row + ix[a]], wzy * wx[a]);
    }
}

__global__ void k_delta(const double *__restrict__ rho, long long m, double inv_mean,
                        float *__restrict__ delta) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) delta[i] = (float)(rho[i] * inv_mean - 1.0);
}

__device__ __forceinline__ void ff_acc(float &hi, float &lo, float v) {
  // float-float accumulation (TwoSum of hi and v, low parts summed)
  const float s = hi + v;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (v - bb);
  hi = s;
  lo += err;
}

// Shared-memory rows are skewed by 4 floats after every 16 (index i lives at
// i + 4 (i / 16)): 16-float blocks read by consecutive lanes then fall on
// distinct banks.
__device__ __forceinline__ int skew(int i) { return i + 4 * (i >> 4); }

constexpr int kStageRowSets = 2;  // rows per lane per stage (smem: occupancy)

// One CTA of G warps: lag column (dy, dz) = cols[blockIdx.x] with lags
// dxmin..dxmax, window dx in [dx0, dx0 + 16 G) (dx0 = dxmin rounded down to
// a multiple of 4, plus 16 G blockIdx.y), rows z in [z0, z1) (blockIdx.z).
// Warp g owns lags dx0 + 16 g .. + 15; its lanes split each row into blocks
// of 16 consecutive x (lpr lanes per row, 32 / lpr rows side by side).  Per
// block a lane loads 16 delta_A and 32 delta_B values (float4 loads) for
// 256 FMAs.  Rows arrive by 16-byte cp.async into two stage buffers, the
// next stage in flight while the current one is summed; FP32 partials are
// folded into float-float accumulators every 8 rows.
__global__ void __launch_bounds__(128, 6) k_lagcorr(const float *__restrict__ delta, int n,
                                                    const int4 *__restrict__ cols, int zslab,
                                                    double *__restrict__ out, int out_stride) {
  extern __shared__ __align__(16) float sm[];
  const int4 col = cols[blockIdx.x];  // (dy, dz, dxmin, dxmax)
  const int dy = col.x, dz = col.y, dxmin = col.z, dxmax = col.w;
  const int G = blockDim.x >> 5;
  const int dx0 = (dxmin >= 0 ? dxmin & ~3 : -((-dxmin + 3) & ~3)) + 16 * G * (int)blockIdx.y;
  if (dx0 > dxmax) return;
  const int z0 = blockIdx.z * zslab, z1 = min(n, z0 + zslab);
  const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lpr = min(32, n >> 4);            // lanes per row
  const int rpw = 32 / lpr;                   // rows side by side in a warp
  const int srows = kStageRowSets * rpw;      // rows per stage
  const int sa_len = skew(n), sb_len = skew(n + 64);
  const int stride = sa_len + sb_len;         // floats per staged row pair
  const int rs = lane / lpr, xl = lane % lpr;
  const bool live = dx0 + 16 * g <= dxmax && dx0 + 16 * g + 15 >= dxmin;
  float hi[16], lo[16], part[16];
#pragma unroll
  for (int k = 0; k < 16; k++) hi[k] = lo[k] = part[k] = 0.0f;
  const int nrows = (z1 - z0) * n;
  const int nstage = (nrows + srows - 1) / srows;
  auto issue = [&](int s) {
    const int r0 = s * srows;
    const int nr = min(srows, nrows - r0);
    float *base = sm + (size_t)(s & 1) * srows * stride;
    int z = z0 + r0 / n, y = r0 - (r0 / n) * n;
    for (int q = 0; q < nr; q++, y++) {
      if (y == n) {
        y = 0;
        z++;
      }
      const int zb = wrapi(z + dz, n), yb = wrapi(y + dy, n);
      const float *A = delta + ((long long)z * n + y) * n;
      const float *B = delta + ((long long)zb * n + yb) * n;
      float *sa = base + q * stride, *sb = sa + sa_len;
      for (int c = threadIdx.x; c < (n >> 2); c += blockDim.x) cp_async16(sa + skew(4 * c), A + 4 * c);
      // sb holds delta_B[(dx0 + i) mod n] at skew(i), i < n + 64
      for (int c = threadIdx.x; c < ((n + 64) >> 2); c += blockDim.x) {
        int xb = 4 * c + dx0;
        while (xb < 0) xb += n;
        while (xb >= n) xb -= n;
        cp_async16(sb + skew(4 * c), B + xb);
      }
    }
    cp_async_commit();
  };
  int since = 0;
  issue(0);
  for (int s = 0; s < nstage; s++) {
    if (s + 1 < nstage) {
      issue(s + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int nr = min(srows, nrows - s * srows);
    const float *base = sm + (size_t)(s & 1) * srows * stride;
    if (live) {
      for (int q = rs; q < nr; q += rpw) {
        const float *sa = base + q * stride, *sb = sa + sa_len;
        for (int xb0 = 16 * xl; xb0 < n; xb0 += 16 * lpr) {
          float a[16], b[32];
          const float *pa = sa + skew(xb0);
          const float *pb0 = sb + skew(xb0 + 16 * g), *pb1 = sb + skew(xb0 + 16 * g + 16);
#pragma unroll
          for (int v = 0; v < 4; v++) {
            *(float4 *)&a[4 * v] = *(const float4 *)(pa + 4 * v);
            *(float4 *)&b[4 * v] = *(const float4 *)(pb0 + 4 * v);
            *(float4 *)&b[16 + 4 * v] = *(const float4 *)(pb1 + 4 * v);
          }
          // part[k] += sum_i delta_A[x + i] delta_B[x + i + dx0 + 16 g + k]
#pragma unroll
          for (int i = 0; i < 16; i++)
#pragma unroll
            for (int k = 0; k < 16; k++) part[k] = fmaf(a[i], b[i + k], part[k]);
        }
        if (++since == 8) {  // fold the FP32 partials every 8 rows
#pragma unroll
          for (int k = 0; k < 16; k++) {
            ff_acc(hi[k], lo[k], part[k]);
            part[k] = 0.0f;
          }
          since = 0;
        }
      }
    }
    __syncthreads();  // the buffer is refilled by the next issue
  }
#pragma unroll
  for (int k = 0; k < 16; k++) ff_acc(hi[k], lo[k], part[k]);
  // reduce the lanes of the warp (all hold lags dx0 + 16 g + k) and add to out
#pragma unroll
  for (int k = 0; k < 16; k++) {
    double v = (double)hi[k] + (double)lo[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int dx = dx0 + 16 * g + k;
    if (live && lane == 0 && dx >= dxmin && dx <= dxmax)
      atomicAdd(&out[(size_t)blockIdx.x * out_stride + (dx - dxmin)], v);
  }
}


// k_lagcorr_w: the lag sums again, one warp per work unit -- a window of at
// most NCH x XL consecutive lags of one (dy, dz) column -- and z slab, for
// grids of n = 32 XL points per row.  No shared memory and no block
// barriers: each lane loads its XL-point block of the row pair's A row and
// of its B row at the window's offset (float4 loads from the L2-resident
// grid; the warps of a block take neighbouring units over the same rows, so
// the A rows are L1 hits for all but one of them), and takes the rest of the
// B window from the next lanes by shuffle, one block per chunk of XL lags:
//   C[w + c XL + j] += sum_i A[x_i] B[x_i + w + c XL + j],  i, j < XL,
// over the blocks of lanes l + c and l + c + 1.  The row loop is compiled
// per number of chunks NC (fixed for a warp), so every chunk, shuffle and
// register is static.  FP32 partials over 32 rows are summed across the warp
// and folded into float-float per lag.
template <int XL, int K, int NC>
__device__ __forceinline__ void lag_rows(const float *__restrict__ delta, int n, int dy, int dz,
                                         int z0, int z1, int xa, int xb, int lane, float (&fh)[(K + 31) / 32],
                                         float (&fl)[(K + 31) / 32]) {
  constexpr int kFold = 32;  // rows per FP32 partial
  float acc[NC * XL];
#pragma unroll
  for (int k = 0; k < NC * XL; k++) acc[k] = 0.0f;
  auto fold = [&]() {
#pragma unroll
    for (int k = 0; k < NC * XL; k++) {
      float v = acc[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == (k & 31)) ff_acc(fh[k >> 5], fl[k >> 5], v);
      acc[k] = 0.0f;
    }
  };
  int since = 0;
  for (int z = z0; z < z1; z++) {
    const int zb = wrapi(z + dz, n);
    const float *A = delta + (long long)z * n * n + xa;
    for (int y = 0; y < n; y++, A += n) {
      const float *B = delta + ((long long)zb * n + wrapi(y + dy, n)) * n;
      float a[XL], own[XL];
#pragma unroll
      for (int q = 0; q < XL / 4; q++) {
        *(float4 *)&a[4 * q] = __ldg((const float4 *)(A + 4 * q));
        const int x = xb + 4 * q;
        *(float4 *)&own[4 * q] = __ldg((const float4 *)(B + (x >= n ? x - n : x)));
      }
      // the window of chunk c: blocks of lanes l + c (cur) and l + c + 1 (nxt)
      float cur[XL], nxt[XL];
#pragma unroll
      for (int t = 0; t < XL; t++) {
        cur[t] = own[t];
        nxt[t] = __shfl_sync(0xffffffffu, own[t], (lane + 1) & 31);
      }
#pragma unroll
      for (int c = 0; c < NC; c++) {
#pragma unroll
        for (int i = 0; i < XL; i++)
#pragma unroll
          for (int j = 0; j < XL; j++)
            acc[c * XL + j] = fmaf(a[i], (i + j < XL) ? cur[i + j] : nxt[i + j - XL], acc[c * XL + j]);
        if (c + 1 < NC) {
#pragma unroll
          for (int t = 0; t < XL; t++) {
            cur[t] = nxt[t];
            nxt[t] = __shfl_sync(0xffffffffu, own[t], (lane + c + 2) & 31);
          }
        }
      }
      if (++since == kFold) {
        fold();
        since = 0;
      }
    }
  }
  fold();
}

template <int XL, int NCH>
__global__ void __launch_bounds__(128) k_lagcorr_w(const float *__restrict__ delta, int n,
                                                   const int4 *__restrict__ units, int nunits,
                                                   const int4 *__restrict__ cols, int zslab,
                                                   double *__restrict__ out, int out_stride) {
  constexpr int K = XL * NCH;        // lags of a window
  constexpr int KF = (K + 31) / 32;  // float-float lag sums per lane
  const int lane = threadIdx.x & 31;
  const int u = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (u >= nunits) return;  // whole warps: no barrier follows
  const int4 un = units[u];  // (column, first lag w, chunks, 0)
  const int4 col = cols[un.x];
  const int w0 = un.y, nch = un.z;
  const int z0 = blockIdx.x * zslab, z1 = min(n, z0 + zslab);
  const int xa = XL * lane;
  // this lane's block of the B row starts at x = xa + w0 (w0 a multiple of 4)
  int xb = xa + w0;
  xb = xb < 0 ? xb + n : (xb >= n ? xb - n : xb);
  float fh[KF], fl[KF];
#pragma unroll
  for (int k = 0; k < KF; k++) fh[k] = fl[k] = 0.0f;
  switch (nch) {
#define LAG_CASE(c)                                                                           \
  case c:                                                                                     \
    if (c <= NCH) lag_rows<XL, K, (c <= NCH ? c : 1)>(delta, n, col.x, col.y, z0, z1, xa, xb, lane, fh, fl); \
    break;
    LAG_CASE(1) LAG_CASE(2) LAG_CASE(3) LAG_CASE(4) LAG_CASE(5)
    LAG_CASE(6) LAG_CASE(7) LAG_CASE(8) LAG_CASE(9) LAG_CASE(10)
#undef LAG_CASE
    default: break;
  }
  const int dxmin = col.z, dxmax = col.w;
#pragma unroll
  for (int k = 0; k < K; k++) {
    const int dx = w0 + k;
    if (lane == (k & 31) && k < nch * XL && dx >= dxmin && dx <= dxmax)
      atomicAdd(&out[(size_t)un.x * out_stride + (dx - dxmin)],
                (double)fh[k >> 5] + (double)fl[k >> 5]);
  }
}

}  // namespace

}  // namespace cute

using namespace cute;

extern "C" cute_status cute_density_grid_xi(cute_ctx *ctx, const double *xyz, const float *w,
                                            int64_t n_obj, double box_L, int32_t ngrid,
                                            const double *edges, int32_t nbins, double *xi_out,
                                            double *lags_out) {
  if (!ctx) return CUTE_E_INVALID;
  ctx->err.clear();
  auto fail = [&](cute_status st, const std::string &m) {
    ctx->err = m;
    return st;
  };
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(CUTE_E_CUDA, "cudaSetDevice");
  if (n_obj < 1 || !xyz || !edges || !xi_out || nbins < 1 || !(box_L > 0) || ngrid < 8 ||
      ngrid > kMaxGrid || ngrid % 32)
    return fail(CUTE_E_INVALID, "bad arguments (ngrid: a multiple of 32 in 32..1024)");
  for (int b = 0; b < nbins; b++)
    if (!(edges[b + 1] > edges[b]) || !(edges[0] >= 0))
      return fail(CUTE_E_INVALID, "edges must be increasing and >= 0");
  const double a = box_L / ngrid;
  const double rmax = edges[nbins];
  if (!(rmax < 0.5 * box_L)) return fail(CUTE_E_INVALID, "r_max must be below L/2");
  const int R = (int)std::floor(rmax / a);  // largest |d| component that can be in range
  if (R < 1) return fail(CUTE_E_INVALID, "r_max must be at least one grid cell");
  // half-ball lag columns (dy, dz) with their dx ranges; a lag is in range
  // when its squared length (in FP64, a^2 |d|^2) is below r_max^2
  std::vector<int4> cols;
  const double r2max = rmax * rmax;
  for (int dz = -R; dz <= R; dz++)
    for (int dy = -R; dy <= R; dy++) {
      if (dz < 0 || (dz == 0 && dy < 0)) continue;  // half space (the other half mirrors)
      const double q = ((double)dy * dy + (double)dz * dz) * a * a;
      if (q >= r2max) continue;
      int xm = 0;
      while ((double)(xm + 1) * (xm + 1) * a * a + q < r2max) xm++;
      const int lo = (dz == 0 && dy == 0) ? 1 : -xm;  // d = 0 excluded, dx > 0 half line
      if (lo > xm) continue;
      cols.push_back(make_int4(dy, dz, lo, xm));
    }
  int maxw = 1;
  for (const int4 &c : cols) maxw = std::max(maxw, c.w - c.z + 1);
  // rows of 128, 256 or 384 points: k_lagcorr_w, one warp per window
  // of K = XL NCH lags of a column (XL = n / 32 points per lane); the
  // windows start at the column's first lag rounded down to a multiple of 4
  const int XL = ngrid / 32;
  const bool warp_kernel = (XL == 4 || XL == 8 || XL == 12);
  const int NCH = XL == 4 ? 10 : (XL == 8 ? 5 : 3);
  std::vector<int4> units;
  if (warp_kernel) {
    for (size_t c = 0; c < cols.size(); c++) {
      const int lo = cols[c].z, hi = cols[c].w;
      const int w0 = lo >= 0 ? lo & ~3 : -((-lo + 3) & ~3);
      for (int w = w0; w <= hi; w += XL * NCH) {
        const int nch = std::min(NCH, (hi - w + XL) / XL);  // chunks reaching hi
        units.push_back(make_int4((int)c, w, nch, 0));
      }
    }
    // longest windows first (blocks start in launch order: the short ones
    // fill in behind them instead of trailing)
    std::stable_sort(units.begin(), units.end(),
                     [](const int4 &p, const int4 &q) { return p.z > q.z; });
  }
  const long long m = (long long)ngrid * ngrid * ngrid;
  const bool dev = [&] {
    cudaPointerAttributes at;
    const bool d = cudaPointerGetAttributes(&at, xyz) == cudaSuccess &&
                   (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    return d;
  }();
  const size_t xb = (size_t)n_obj * 3 * sizeof(double), wb = w ? (size_t)n_obj * sizeof(float) : 0;
  const size_t ob = cols.size() * (size_t)maxw * sizeof(double);
  const size_t need = 256 + m * sizeof(double) + m * sizeof(float) + cols.size() * sizeof(int4) +
                      ob + (dev ? 0 : xb + wb) + units.size() * sizeof(int4) + 2048;
  char *buf = nullptr;
  if (cudaMalloc(&buf, need) != cudaSuccess) return fail(CUTE_E_OOM, "cudaMalloc");
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  int *d_bad = (int *)buf;
  double *d_rho = (double *)(buf + 256);
  float *d_delta = (float *)((char *)d_rho + al(m * sizeof(double)));
  int4 *d_cols = (int4 *)((char *)d_delta + al(m * sizeof(float)));
  double *d_out = (double *)((char *)d_cols + al(cols.size() * sizeof(int4)));
  const double *d_xyz = xyz;
  const float *d_w = w;
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
  int4 *d_units = (int4 *)((char *)d_out + al(ob));
  if (!dev) {
    char *p = (char *)d_units + al(units.size() * sizeof(int4));
    d_xyz = (const double *)p;
    d_w = w ? (const float *)(p + al(xb)) : nullptr;
    if (e == cudaSuccess) e = cudaMemcpyAsync((void *)d_xyz, xyz, xb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && w) e = cudaMemcpyAsync((void *)d_w, w, wb, cudaMemcpyHostToDevice, st);
  } else if (w) {
    cudaPointerAttributes at;
    const bool wd = cudaPointerGetAttributes(&at, w) == cudaSuccess &&
                    (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (!wd) {
      cudaFree(buf);
      return fail(CUTE_E_INVALID, "xyz and w must both be device or both host memory");
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(d_rho, 0, m * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_out, 0, ob, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_cols, cols.data(), cols.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !units.empty())
    e = cudaMemcpyAsync(d_units, units.data(), units.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
  // total weight for the mean density
  double wsum = (double)n_obj;
  if (w) {
    std::vector<float> hw(n_obj);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hw.data(), d_w, wb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    wsum = 0;
    for (float v : hw) wsum += v;
  }
  if (e == cudaSuccess && !(wsum > 0)) {
    cudaFree(buf);
    return fail(CUTE_E_INVALID, "total weight must be positive");
  }
  if (e == cudaSuccess) {
    k_tsc<<<(unsigned)((n_obj + 255) / 256), 256, 0, st>>>(d_xyz, d_w, n_obj, ngrid, 1.0 / a, d_rho,
                                                           d_bad, box_L);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_delta<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(d_rho, m, (double)m / wsum, d_delta);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && warp_kernel) {
    // four warps (units) per block; z slabs of n / 16 rows
    const int zslab = std::max(1, ngrid / 16);
    // grid x: z slabs, y: groups of four units (the same rows for the four)
    dim3 grid((unsigned)((ngrid + zslab - 1) / zslab), (unsigned)((units.size() + 3) / 4));
    ctx->stats = cute_stats{};
    cudaMemsetAsync(ctx->d_ticket, 0, kCounterWords * sizeof(unsigned long long), st);
    ctx->stats.launches = 1;
    ctx->stats.blocks = (int)(grid.x * grid.y);
    ctx->stats.warps_per_block = 4;
    if (ctx->timing) cudaEventRecord(ctx->ev0, st);
    const int nu = (int)units.size();
    if (XL == 4) k_lagcorr_w<4, 10><<<grid, 128, 0, st>>>(d_delta, ngrid, d_units, nu, d_cols, zslab, d_out, maxw);
    else if (XL == 8) k_lagcorr_w<8, 5><<<grid, 128, 0, st>>>(d_delta, ngrid, d_units, nu, d_cols, zslab, d_out, maxw);
    else k_lagcorr_w<12, 3><<<grid, 128, 0, st>>>(d_delta, ngrid, d_units, nu, d_cols, zslab, d_out, maxw);
    if (ctx->timing) cudaEventRecord(ctx->ev1, st);
    e = cudaGetLastError();
  } else if (e == cudaSuccess) {
    const int zslab = std::max(1, ngrid / 8);
    // 16 lags per warp, as many warps as the widest column's window needs
    // (it starts at dxmin rounded down to a multiple of 4); warps past a
    // narrower column's end only help staging
    const int wmax = maxw + 3;
    const int G = std::min(4, (wmax + 15) / 16);
    dim3 grid((unsigned)cols.size(), (unsigned)((wmax + 16 * G - 1) / (16 * G)),
              (unsigned)((ngrid + zslab - 1) / zslab));
    auto skew_h = [](int i) { return i + 4 * (i >> 4); };
    const int srows = kStageRowSets * (32 / std::min(32, ngrid / 16));
    const size_t smem = (size_t)2 * srows * (skew_h(ngrid) + skew_h(ngrid + 64)) * sizeof(float);
    if (smem > 48 * 1024)
      e = cudaFuncSetAttribute(k_lagcorr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      ctx->stats = cute_stats{};
      cudaMemsetAsync(ctx->d_ticket, 0, kCounterWords * sizeof(unsigned long long), st);
      ctx->stats.launches = 1;
      ctx->stats.blocks = (int)(grid.x * grid.y * grid.z);
      ctx->stats.warps_per_block = G;
      if (ctx->timing) cudaEventRecord(ctx->ev0, st);
      k_lagcorr<<<grid, 32 * G, smem, st>>>(d_delta, ngrid, d_cols, zslab, d_out, maxw);
      if (ctx->timing) cudaEventRecord(ctx->ev1, st);
      e = cudaGetLastError();
    }
  }
  std::vector<double> C(cols.size() * (size_t)maxw);
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(C.data(), d_out, ob, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) return fail(CUTE_E_CUDA, cudaGetErrorString(e));
  if (bad) return fail(CUTE_E_INVALID, "positions must lie in [0, L)");
  // bin the lags: half-open bins on the squared separation a^2 |d|^2
  std::vector<double> E2(nbins + 1), sum(nbins, 0.0), cnt(nbins, 0.0);
  for (int b = 0; b <= nbins; b++) E2[b] = edges[b] * edges[b];
  for (size_t c = 0; c < cols.size(); c++) {
    const int4 col = cols[c];
    for (int dx = col.z; dx <= col.w; dx++) {
      const double r2 = ((double)dx * dx + (double)col.x * col.x + (double)col.y * col.y) * a * a;
      if (r2 < E2[0] || r2 >= E2[nbins]) continue;
      const int b = (int)(std::upper_bound(E2.begin(), E2.end(), r2) - E2.begin()) - 1;
      sum[b] += C[c * maxw + (dx - col.z)];
      cnt[b] += 1.0;
    }
  }
  for (int b = 0; b < nbins; b++) {
    xi_out[b] = cnt[b] > 0 ? sum[b] / (cnt[b] * (double)m) : NAN;
    if (lags_out) lags_out[b] = cnt[b];
  }
  return CUTE_OK;
}

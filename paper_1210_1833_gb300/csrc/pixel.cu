// pixel.cu -- pixel maps of angular catalogs (Sec. 3.4.2).
//
// For w(theta) at scales well above a pixel, the catalog is binned into an
// equal-area pixel map and the pixels are correlated instead of the objects,
// each pixel weighted by the objects it holds; the weighted angular count of
// the pixel centres then stands in for the object count.  The paper does not
// fix the pixelisation; the HEALPix RING scheme (Gorski et al. 2005, ApJ 622,
// 759) is used here: 12 nside^2 equal-area pixels on iso-latitude rings,
// rings 1..nside-1 and 3nside+1..4nside-1 in the polar caps (4i pixels on
// the i-th ring from a pole), rings nside..3nside in the equatorial belt
// (4 nside pixels each, every other ring shifted by half a pixel).
#include "cute_internal.h"

#include <cmath>
#include <string>

namespace cute {

namespace {

constexpr double kPi = 3.14159265358979323846;

// pixel of the unit vector (x, y, z): z = cos(theta), phi = atan2(y, x)
__device__ long long ang2pix_ring(long long ns, double x, double y, double z) {
  double phi = atan2(y, x);
  if (phi < 0.0) phi += 2.0 * kPi;
  const double tt = fmod(phi / (0.5 * kPi), 4.0);  // in [0, 4)
  const double za = fabs(z);
  const long long npix = 12 * ns * ns, ncap = 2 * ns * (ns - 1);
  if (za <= 2.0 / 3.0) {
    // equatorial belt: indices of the two edge lines through the point
    const double t1 = ns * (0.5 + tt), t2 = ns * z * 0.75;
    const long long jp = (long long)floor(t1 - t2), jm = (long long)floor(t1 + t2);
    const long long ir = ns + 1 + jp - jm;  // 1 .. 2 ns + 1, from the ring at z = 2/3
    const long long kshift = 1 - (ir & 1);
    long long ip = (jp + jm - ns + kshift + 1) / 2;
    ip = ip % (4 * ns);
    if (ip < 0) ip += 4 * ns;
    return ncap + (ir - 1) * 4 * ns + ip;
  }
  // polar caps
  const double tp = tt - floor(tt);
  const double tmp = ns * sqrt(3.0 * (1.0 - za));
  const long long jp = (long long)floor(tp * tmp), jm = (long long)floor((1.0 - tp) * tmp);
  const long long ir = jp + jm + 1;  // 1 .. ns, from the nearest pole
  long long ip = (long long)floor(tt * ir);
  ip = ip % (4 * ir);
  return z > 0.0 ? 2 * ir * (ir - 1) + ip : npix - 2 * ir * (ir + 1) + ip;
}

__device__ long long isqrt_ll(long long v) {
  long long r = (long long)sqrt((double)v);
  while (r * r > v) r--;
  while ((r + 1) * (r + 1) <= v) r++;
  return r;
}

// centre of pixel p as a unit vector
__device__ void pix2vec_ring(long long ns, long long p, double *v) {
  const long long npix = 12 * ns * ns, ncap = 2 * ns * (ns - 1);
  double z, phi;
  if (p < ncap) {  // north cap: ring i holds pixels 2i(i-1) .. 2i(i+1)-1
    const long long i = (1 + isqrt_ll(1 + 2 * p)) / 2;
    const long long j = p + 1 - 2 * i * (i - 1);  // 1 .. 4i
    z = 1.0 - (double)(i * i) / (3.0 * (double)ns * (double)ns);
    phi = (j - 0.5) * kPi / (2.0 * i);
  } else if (p < npix - ncap) {  // equatorial belt
    const long long q = p - ncap;
    const long long i = q / (4 * ns) + ns;  // ring from the north pole, ns .. 3 ns
    const long long j = q % (4 * ns) + 1;
    const double shift = ((i + ns) & 1) ? 1.0 : 0.5;
    z = (double)(2 * ns - i) * 2.0 / (3.0 * (double)ns);
    phi = (j - shift) * kPi / (2.0 * ns);
  } else {  // south cap, counted back from the last pixel
    const long long q = npix - p;
    const long long i = (1 + isqrt_ll(2 * q - 1)) / 2;
    const long long j = 4 * i + 1 - (q - 2 * i * (i - 1));
    z = -1.0 + (double)(i * i) / (3.0 * (double)ns * (double)ns);
    phi = (j - 0.5) * kPi / (2.0 * i);
  }
  const double st = sqrt((1.0 - z) * (1.0 + z));
  double sp, cp;
  sincos(phi, &sp, &cp);
  v[0] = st * cp;
  v[1] = st * sp;
  v[2] = z;
}

__global__ void k_pixel_map(const double *__restrict__ xyz, const float *__restrict__ w,
                            long long n, long long ns, double *__restrict__ map,
                            int *__restrict__ bad) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  const double r2 = x * x + y * y + z * z;
  if (!(fabs(r2 - 1.0) <= 1e-6)) {  // not a unit vector (NaN included)
    atomicExch(bad, 1);
    return;
  }
  const long long p = ang2pix_ring(ns, x, y, z);
  atomicAdd(&map[p], w ? (double)w[i] : 1.0);
}

__global__ void k_pixel_centres(const long long *__restrict__ pix, long long m, long long ns,
                                double *__restrict__ xyz, int *__restrict__ bad) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const long long p = pix[i];
  if (p < 0 || p >= 12 * ns * ns) {
    atomicExch(bad, 1);
    xyz[3 * i] = xyz[3 * i + 1] = xyz[3 * i + 2] = 0.0;
    return;
  }
  pix2vec_ring(ns, p, xyz + 3 * i);
}

bool on_device(const void *p) {
  cudaPointerAttributes at;
  const bool d = cudaPointerGetAttributes(&at, p) == cudaSuccess &&
                 (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  return d;
}

// Runs `launch(device pointers...)` with host arrays staged through one
// device buffer: in-arrays copied in, out-array copied back.
struct Stage {
  char *buf = nullptr;
  ~Stage() { cudaFree(buf); }
};

}  // namespace

}  // namespace cute

using namespace cute;

extern "C" cute_status cute_pixel_map(cute_ctx *ctx, const double *xyz, const float *w, int64_t n,
                                      int32_t nside, double *map) {
  if (!ctx) return CUTE_E_INVALID;
  ctx->err.clear();
  auto fail = [&](cute_status st, const std::string &m) {
    ctx->err = m;
    return st;
  };
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(CUTE_E_CUDA, "cudaSetDevice");
  if (n < 0 || (n > 0 && !xyz) || !map || nside < 1 || nside > 8192 || (nside & (nside - 1)))
    return fail(CUTE_E_INVALID, "bad arguments (nside: a power of 2 up to 8192)");
  const bool dev = on_device(map);
  if ((n > 0 && on_device(xyz) != dev) || (w && on_device(w) != dev))
    return fail(CUTE_E_INVALID, "xyz, w and map must all be device or all host memory");
  const long long npix = 12LL * nside * nside;
  const size_t mb = (size_t)npix * sizeof(double), xb = (size_t)n * 3 * sizeof(double),
               wb = w ? (size_t)n * sizeof(float) : 0;
  Stage s;
  const size_t need = 256 + (dev ? 0 : mb + xb + wb + 512);
  if (cudaMalloc(&s.buf, need) != cudaSuccess) return fail(CUTE_E_OOM, "cudaMalloc");
  int *d_bad = (int *)s.buf;
  const double *d_xyz = xyz;
  const float *d_w = w;
  double *d_map = map;
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
  if (!dev) {
    char *p = s.buf + 256;
    d_map = (double *)p;
    d_xyz = (const double *)(p + ((mb + 255) & ~(size_t)255));
    d_w = w ? (const float *)((const char *)d_xyz + ((xb + 255) & ~(size_t)255)) : nullptr;
    if (e == cudaSuccess && n > 0)
      e = cudaMemcpyAsync((void *)d_xyz, xyz, xb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && w) e = cudaMemcpyAsync((void *)d_w, w, wb, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(d_map, 0, mb, st);
  if (e == cudaSuccess && n > 0) {
    k_pixel_map<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_xyz, d_w, n, nside, d_map, d_bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(map, d_map, mb, cudaMemcpyDeviceToHost, st);
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(CUTE_E_CUDA, cudaGetErrorString(e));
  if (bad) return fail(CUTE_E_INVALID, "positions must be unit vectors (|x|^2 within 1e-6 of 1)");
  return CUTE_OK;
}

extern "C" cute_status cute_pixel_centres(cute_ctx *ctx, int32_t nside, const int64_t *pix,
                                          int64_t m, double *xyz) {
  if (!ctx) return CUTE_E_INVALID;
  ctx->err.clear();
  auto fail = [&](cute_status st, const std::string &msg) {
    ctx->err = msg;
    return st;
  };
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(CUTE_E_CUDA, "cudaSetDevice");
  if (m < 0 || (m > 0 && (!pix || !xyz)) || nside < 1 || nside > 8192 || (nside & (nside - 1)))
    return fail(CUTE_E_INVALID, "bad arguments (nside: a power of 2 up to 8192)");
  if (m == 0) return CUTE_OK;
  const bool dev = on_device(pix);
  if (on_device(xyz) != dev) return fail(CUTE_E_INVALID, "pix and xyz must both be device or host memory");
  const size_t pb = (size_t)m * sizeof(int64_t), xb = (size_t)m * 3 * sizeof(double);
  Stage s;
  if (cudaMalloc(&s.buf, 256 + (dev ? 0 : pb + xb + 256)) != cudaSuccess)
    return fail(CUTE_E_OOM, "cudaMalloc");
  int *d_bad = (int *)s.buf;
  const long long *d_pix = (const long long *)pix;
  double *d_xyz = xyz;
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
  if (!dev) {
    d_pix = (const long long *)(s.buf + 256);
    d_xyz = (double *)(s.buf + 256 + ((pb + 255) & ~(size_t)255));
    if (e == cudaSuccess) e = cudaMemcpyAsync((void *)d_pix, pix, pb, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) {
    k_pixel_centres<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(d_pix, m, nside, d_xyz, d_bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(xyz, d_xyz, xb, cudaMemcpyDeviceToHost, st);
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(CUTE_E_CUDA, cudaGetErrorString(e));
  if (bad) return fail(CUTE_E_INVALID, "pixel index outside 0 .. 12 nside^2 - 1");
  return CUTE_OK;
}

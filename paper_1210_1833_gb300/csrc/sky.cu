// sky.cu -- comoving positions from sky coordinates.
//
// Catalogs of surveys come as (RA, Dec, z).  The 3-D measures need the
// comoving position chi(z) n, with chi the radial comoving distance of
// Sec. 2.1 and n the unit vector towards (RA, Dec); the angular measure
// projects every object onto the unit sphere (Sec. 3.4.2), i.e. n alone.
//
// chi(z) = (c / H0) integral_0^z dz' / E(z'), c / H0 = 2997.92458 Mpc/h,
// E(z)^2 = Om (1+z)^3 + Ok (1+z)^2 + OL (1+z)^(3 (1 + w)), Ok = 1 - Om - OL.
// The host tabulates chi on a uniform grid of z (each interval integrated
// with 8-point Gauss-Legendre quadrature, FP64) together with its derivative
// (c/H0)/E; the kernel interpolates with cubic Hermite polynomials, whose
// error for this smooth integrand is far below 1e-12 relative at the grid
// spacing used.
#include "cute_internal.h"

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace cute {

namespace {

constexpr double kCoverH0 = 2997.92458;  // c / H0 in Mpc/h
constexpr double kZMax = 20.0;            // table range
constexpr int kTable = 40000;             // intervals: dz = 5e-4

struct Cosmo {
  double om, ok, ol, w;
  double E(double z) const {
    const double a = 1.0 + z;
    const double de = w == -1.0 ? 1.0 : std::pow(a, 3.0 * (1.0 + w));
    return std::sqrt(om * a * a * a + ok * a * a + ol * de);
  }
};

// 8-point Gauss-Legendre nodes and weights on [-1, 1]
const double kGx[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290,
                       -0.1834346424956498, 0.1834346424956498,  0.5255324099163290,
                       0.7966664774136267,  0.9602898564975363};
const double kGw[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873,
                       0.3626837833783620, 0.3626837833783620, 0.3137066458778873,
                       0.2223810344533745, 0.1012285362903763};

__global__ void k_sky_to_xyz(const double *__restrict__ ra, const double *__restrict__ dec,
                             const double *__restrict__ z, long long n,
                             const double2 *__restrict__ tab, double dz, double *__restrict__ xyz,
                             int *__restrict__ bad) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double sa, ca, sd, cd;
  sincospi(ra[i] / 180.0, &sa, &ca);
  sincospi(dec[i] / 180.0, &sd, &cd);
  double r = 1.0;
  if (z) {
    const double zi = z[i];
    if (!(zi >= 0.0 && zi <= kZMax)) {  // also catches NaN
      atomicExch(bad, 1);
      r = 0.0;
    } else {
      // cubic Hermite on [z_k, z_k+1] from chi and dchi/dz = (c/H0)/E
      int k = (int)(zi / dz);
      k = min(k, kTable - 1);
      const double t = zi / dz - k;
      const double2 a = tab[k], b = tab[k + 1];  // (chi, dchi/dz)
      const double t2 = t * t, t3 = t2 * t;
      const double h00 = 2.0 * t3 - 3.0 * t2 + 1.0, h10 = t3 - 2.0 * t2 + t;
      const double h01 = -2.0 * t3 + 3.0 * t2, h11 = t3 - t2;
      r = h00 * a.x + h10 * dz * a.y + h01 * b.x + h11 * dz * b.y;
    }
  }
  xyz[3 * i] = r * cd * ca;
  xyz[3 * i + 1] = r * cd * sa;
  xyz[3 * i + 2] = r * sd;
}

}  // namespace

}  // namespace cute

using namespace cute;

extern "C" cute_status cute_sky_to_xyz(cute_ctx *ctx, const double *ra, const double *dec,
                                       const double *z, int64_t n, const cute_cosmology *cosmo,
                                       double *xyz) {
  if (!ctx) return CUTE_E_INVALID;
  ctx->err.clear();
  auto fail = [&](cute_status st, const std::string &m) {
    ctx->err = m;
    return st;
  };
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(CUTE_E_CUDA, "cudaSetDevice");
  if (n < 0 || (n > 0 && (!ra || !dec || !xyz))) return fail(CUTE_E_INVALID, "bad arguments");
  if (z && !cosmo) return fail(CUTE_E_INVALID, "redshifts need a cosmology");
  if (n == 0) return CUTE_OK;
  Cosmo c{0, 0, 0, -1};
  if (z) {
    c.om = cosmo->omega_m;
    c.ol = cosmo->omega_l;
    c.w = cosmo->w0;
    c.ok = 1.0 - c.om - c.ol;
    if (!(c.om >= 0) || !(c.ol >= 0) || !std::isfinite(c.w))
      return fail(CUTE_E_INVALID, "cosmology: omega_m, omega_l >= 0 and finite w0 required");
    for (int k = 0; k <= 64; k++)
      if (!(c.E(kZMax * k / 64.0) > 0)) return fail(CUTE_E_INVALID, "cosmology: E(z) <= 0 below z = 20");
  }
  // where the arrays live: all on the device, or all on the host
  auto on_device = [](const void *p) {
    cudaPointerAttributes at;
    const bool d = cudaPointerGetAttributes(&at, p) == cudaSuccess &&
                   (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    return d;
  };
  const bool dev = on_device(ra);
  if (on_device(dec) != dev || on_device(xyz) != dev || (z && on_device(z) != dev))
    return fail(CUTE_E_INVALID, "ra, dec, z and xyz must all be device or all host memory");
  const size_t nb = (size_t)n * sizeof(double);
  std::vector<double2> tab(z ? kTable + 1 : 1);
  const double dz = kZMax / kTable;
  if (z) {
    tab[0] = make_double2(0.0, kCoverH0 / c.E(0.0));
    double chi = 0.0;
    for (int k = 0; k < kTable; k++) {
      const double z0 = k * dz, zm = z0 + 0.5 * dz;
      double s = 0.0;
      for (int g = 0; g < 8; g++) s += kGw[g] / c.E(zm + 0.5 * dz * kGx[g]);
      chi += kCoverH0 * 0.5 * dz * s;
      tab[k + 1] = make_double2(chi, kCoverH0 / c.E(z0 + dz));
    }
  }
  // device buffers: table, flag, and (for host arrays) staging copies
  char *buf = nullptr;
  const size_t tb = tab.size() * sizeof(double2);
  const size_t stage = dev ? 0 : (z ? 3 : 2) * nb + 3 * nb;
  if (cudaMalloc(&buf, tb + 256 + stage) != cudaSuccess) return fail(CUTE_E_OOM, "cudaMalloc");
  double2 *d_tab = (double2 *)buf;
  int *d_bad = (int *)(buf + tb);
  const double *d_ra = ra, *d_dec = dec, *d_z = z;
  double *d_xyz = xyz;
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(d_tab, tab.data(), tb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
  if (e == cudaSuccess && !dev) {
    double *s = (double *)(buf + tb + 256);
    d_ra = s;
    d_dec = s + n;
    d_xyz = s + 2 * n;
    d_z = z ? s + 5 * n : nullptr;
    e = cudaMemcpyAsync((void *)d_ra, ra, nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync((void *)d_dec, dec, nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && z) e = cudaMemcpyAsync((void *)d_z, z, nb, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) {
    k_sky_to_xyz<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_ra, d_dec, d_z, n, d_tab, dz,
                                                              d_xyz, d_bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(xyz, d_xyz, 3 * nb, cudaMemcpyDeviceToHost, st);
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) return fail(CUTE_E_CUDA, cudaGetErrorString(e));
  if (bad) return fail(CUTE_E_INVALID, "redshifts must lie in [0, 20]");
  return CUTE_OK;
}

// GPU check of the error bounds the counting kernels' FP32 binning assumes
// for two hardware approximations (PTX ISA): lg2.approx.ftz.f32 within
// 2^-21 + 2^-22 |log2 x| of log2(x) (an absolute part, and about two ulp of
// the FP32 result, whose own rounding grows with |log2 x|; the log-spaced
// binning) and rsqrt.approx.ftz.f32 within 2^-22.9 of 1/sqrt(x) (relative;
// every arithmetic binning).  Every FP32 mantissa of every exponent in
// [2^-60, 2^70) is evaluated and compared with the FP64 functions; prints
// "lg2_max_abs lg2_max_over_bound rsqrt_max_rel" and exits 0.
//
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 approx_bound_check.cu
#include <cstdio>
#include <cstdint>
#include <cmath>

__device__ __forceinline__ float lg2_hw(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_hw(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// non-negative doubles order like their bit patterns
__device__ void max_bits(unsigned long long *m, double v) {
  atomicMax(m, (unsigned long long)__double_as_longlong(v));
}

// thread i covers the mantissas [i * 64, i * 64 + 64) of exponent e0 + blockIdx.y
__global__ void k_check(int e0, unsigned long long *out) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;  // < 2^23 / 64
  const int e = e0 + (int)blockIdx.y;                        // unbiased exponent
  double lg = 0, lgn = 0, rs = 0;
  for (uint32_t k = 0; k < 64; k++) {
    const uint32_t m = t * 64u + k;
    const float x = __uint_as_float(((uint32_t)(e + 127) << 23) | m);
    const double xd = (double)x;
    const double l = log2(xd), el = fabs((double)lg2_hw(x) - l);
    lg = fmax(lg, el);
    lgn = fmax(lgn, el / (0x1p-21 + 0x1p-22 * fabs(l)));
    const double r = 1.0 / sqrt(xd);
    rs = fmax(rs, fabs((double)rsqrt_hw(x) - r) / r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lg = fmax(lg, __shfl_xor_sync(0xffffffffu, lg, o));
    lgn = fmax(lgn, __shfl_xor_sync(0xffffffffu, lgn, o));
    rs = fmax(rs, __shfl_xor_sync(0xffffffffu, rs, o));
  }
  if ((threadIdx.x & 31) == 0) {
    max_bits(&out[0], lg);
    max_bits(&out[1], rs);
    max_bits(&out[2], lgn);
  }
}

int main() {
  unsigned long long *d = nullptr, h[3] = {0, 0, 0};
  if (cudaMalloc(&d, sizeof(h)) != cudaSuccess) return 2;
  cudaMemset(d, 0, sizeof(h));
  const int e0 = -60, ne = 130;                    // 2^-60 .. 2^70: normal FP32 values
  const dim3 grid((1u << 23) / 64 / 256, ne), block(256);
  k_check<<<grid, block>>>(e0, d);
  if (cudaDeviceSynchronize() != cudaSuccess) return 3;
  cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  double lg, rs, lgn;
  static_assert(sizeof(double) == sizeof(unsigned long long), "");
  __builtin_memcpy(&lg, &h[0], 8);
  __builtin_memcpy(&rs, &h[1], 8);
  __builtin_memcpy(&lgn, &h[2], 8);
  std::printf("%.6e %.6e %.6e\n", lg, lgn, rs);
  return 0;
}

// Device self-test of the integer-unit float <-> double conversions (fp_convert.cuh)
// against the hardware conversions.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.h"
#include "fp_convert.cuh"

namespace {

// every binary32 pattern: f2d_int must equal the hardware conversion bit for bit (NaN:
// both NaN; a subnormal input gives the signed zero)
__global__ void k_check_f2d(unsigned long long* bad) {
  unsigned long long n = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (1ull << 32); i += stride) {
    const float f = __uint_as_float((uint32_t)i);
    const double a = yt::f2d_int(f), b = (double)f;
    const bool sub = ((uint32_t)i & 0x7F800000u) == 0u;
    const bool same = (a != a && b != b) ||
                      (__double_as_longlong(a) == __double_as_longlong(b)) ||
                      (sub && __double_as_longlong(a) == (long long)((uint64_t)(i & 0x80000000u) << 32));
    n += same ? 0 : 1;
  }
  if (n) atomicAdd(bad, n);
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {   // splitmix64 finaliser
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// doubles whose binary32 rounding is normal or overflows, random fractions, with every
// 8th value a tie (dropped bits exactly one half) and the specials; results the hardware
// rounds to a subnormal float are accepted as signed zeros (flush to zero)
__global__ void k_check_d2f(unsigned long long* bad, uint64_t count) {
  unsigned long long n = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const uint64_t h = mix64(i + 1);
    const uint64_t sign = h & 0x8000000000000000ull;
    const uint64_t exp = 1023ull - 127 + (mix64(h) % 260);         // up to overflow
    uint64_t frac = h & 0xFFFFFFFFFFFFFull;
    if ((i & 7) == 0) frac = (frac & ~0x1FFFFFFFull) | 0x10000000ull;
    double d = __longlong_as_double((long long)(sign | (exp << 52) | frac));
    if (i < 6) {
      const double sp[6] = {0.0, -0.0, __longlong_as_double(0x7FF0000000000000ll),
                            __longlong_as_double((long long)0xFFF0000000000000ull),
                            __longlong_as_double(0x7FF8000000000001ll), 3.4028235677973366e38};
      d = sp[i];
    }
    const float a = yt::d2f_int(d), b = __double2float_rn(d);
    const uint32_t ua = __float_as_uint(a), ub = __float_as_uint(b);
    const bool sub = (ub & 0x7F800000u) == 0u;                      // zero or subnormal
    const bool same = (a != a && b != b) || ua == ub || (sub && ua == (ub & 0x80000000u));
    n += same ? 0 : 1;
  }
  if (n) atomicAdd(bad, n);
}

}  // namespace

extern "C" yt_status yt_selftest_conversions(int64_t* f2d_mismatches, int64_t* d2f_mismatches) {
  return yt::guarded([&] {
    YT_REQUIRE(f2d_mismatches && d2f_mismatches, YT_ERR_INVALID, "null argument");
    unsigned long long* d = nullptr;
    yt::cuda_check(cudaMalloc(&d, 2 * sizeof(unsigned long long)), "cudaMalloc");
    cudaError_t e = cudaMemset(d, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) {
      k_check_f2d<<<1024, 256>>>(d);
      k_check_d2f<<<1024, 256>>>(d + 1, 1ull << 28);
      e = cudaGetLastError();
    }
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    yt::cuda_check(e, "conversion self-test");
    *f2d_mismatches = (int64_t)h[0];
    *d2f_mismatches = (int64_t)h[1];
  });
}

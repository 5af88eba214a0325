// Device self-check of the integer binary32 <-> binary64 conversions (fpconv.cuh) against
// the hardware conversion instructions.
#include <cuda_runtime.h>

#include "fpconv.cuh"
#include "kpsb_internal.cuh"

namespace kpsb {

__device__ __forceinline__ unsigned long long cc_mix(unsigned long long z) {  // splitmix64 finaliser
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ bool same_f64(double a, double b) {
  return __double_as_longlong(a) == __double_as_longlong(b) || (a != a && b != b);
}
__device__ __forceinline__ bool same_f32(float a, float b) {
  return __float_as_uint(a) == __float_as_uint(b) || (a != a && b != b);
}

// Every binary32 pattern through f2d_bits; n_random binary64 patterns through d2f_rn_bits,
// their exponents spread over the binary32 subnormal, normal and overflow range (plus binary64
// zeros, subnormals, infinities and NaNs) and their dropped 29 bits forced, for a quarter of
// them each, to exactly half, half - 1 and half + 1 of the kept bit.
__global__ void conversion_check_kernel(unsigned long long n_random, unsigned long long seed,
                                        unsigned long long* __restrict__ bad) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long nb = 0;
  for (unsigned long long i = t0; i < (1ull << 32); i += stride) {
    const float f = __uint_as_float((unsigned)i);
    nb += same_f64(f2d_bits(f), (double)f) ? 0 : 1;
  }
  for (unsigned long long i = t0; i < n_random; i += stride) {
    const unsigned long long h = cc_mix(seed + 0x9e3779b97f4a7c15ull * (i + 1));
    const unsigned long long h2 = cc_mix(h);
    unsigned long long ex;
    switch (h2 & 15u) {
      case 0: ex = 0; break;                                 // binary64 zero / subnormal
      case 1: ex = 0x7ff; break;                             // infinity / NaN
      case 2: ex = (h2 >> 8) & 0x7ff; break;                 // anywhere
      default: ex = 896 - 30 + ((h2 >> 8) % 300); break;     // around the binary32 range
    }
    unsigned long long fr = h & 0xfffffffffffffull;
    switch ((h2 >> 4) & 3u) {
      case 0: fr = (fr & ~0x1fffffffull) | 0x10000000ull; break;
      case 1: fr = (fr & ~0x1fffffffull) | 0x0fffffffull; break;
      case 2: fr = (fr & ~0x1fffffffull) | 0x10000001ull; break;
      default: break;
    }
    if (ex == 0x7ff && ((h2 >> 6) & 1u)) fr = 0;  // half of them infinities
    const unsigned long long bits = (h & 0x8000000000000000ull) | (ex << 52) | fr;
    const double d = __longlong_as_double((long long)bits);
    nb += same_f32(d2f_rn_bits(d), __double2float_rn(d)) ? 0 : 1;
  }
  if (nb) atomicAdd(bad, nb);
}

}  // namespace kpsb

using namespace kpsb;

extern "C" kpsb_status kpsb_conversion_check(unsigned long long n_random, unsigned long long seed,
                                             unsigned long long* mismatches) {
  clear_error();
  KPSB_REQUIRE(mismatches, "null pointer");
  int dev = 0, sms = 0;
  KPSB_TRY_CUDA(cudaGetDevice(&dev));
  KPSB_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  unsigned long long* d = nullptr;
  KPSB_TRY_CUDA(cudaMalloc((void**)&d, sizeof(unsigned long long)));
  cudaError_t e = cudaMemset(d, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) {
    conversion_check_kernel<<<sms * 8, 256>>>(n_random, seed, d);
    e = cudaGetLastError();
    count_launch();
  }
  if (e == cudaSuccess) e = cudaMemcpy(mismatches, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    set_error("conversion check: %s", cudaGetErrorString(e));
    return KPSB_ECUDA;
  }
  return KPSB_OK;
}

// Shared helpers of the kpsb CUDA library (sm_103a): status/error plumbing, launch
// checks, deterministic grid reductions, warp/block sums.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/kpsb.h"

namespace kpsb {

// Thread-local last-error message (kpsb_last_error).
void set_error(const char* fmt, ...);
void clear_error();
// Process-wide count of kernels launched by this library (kpsb_kernel_launches).  While
// this thread captures a CUDA graph, launches are not counted at capture time; the graph's
// owner counts the kernels that actually ran.
void count_launch(long long n = 1);
void set_capture_mode(bool on);
void trace(cudaStream_t st, const char* phase);
bool gemm_timing_enabled();
// CUDA-event timing (kpsb_gemm_timing / kpsb_timer_stats) by category: the
// Kronecker-sum GEMM applies and the split Bregman vector kernels.
enum TimerCategory {
  TIMER_KP_APPLY = 0,  // one KP apply of a batch
  TIMER_SB_ZZ = 1,     // ||z||^2 (CGLS steps 3-4)
  TIMER_SB_X = 2,      // x, r updates and RC_CGLS (steps 5-6)
  TIMER_SB_F = 3,      // f = Ahat^T r and its norm (steps 7-9)
  TIMER_SB_W = 4,      // w = f + delta w (step 10)
  TIMER_SB_OUTER = 5,  // outer-step kernels: start of an outer step, shrinkage
  TIMER_RA = 6,        // R(A) products of the TSVD (index map or explicit matrix)
  TIMER_REORTH = 7,    // CGS2 reorthogonalisation of the EGKB bases
  TIMER_QR = 8,        // SVQB orthonormalisation of the RSVD blocks
  TIMER_EGKB_BLOCK = 9,  // one-block EGKB recurrence launches (all problems of a batch)
  TIMER_CATEGORIES = 10
};
int timer_begin(cudaStream_t st);
void timer_end(int slot, cudaStream_t st, int cat, double flops, int launches);
// Sets the work value of a recorded slot once it is known (counted on the device).
void timer_set_value(int slot, double v);
int gemm_timer_begin(cudaStream_t st);
void gemm_timer_end(int slot, cudaStream_t st, double flops, int launches);

struct Status {
  kpsb_status code;
};

#define KPSB_TRY_CUDA(expr)                                                            \
  do {                                                                                 \
    cudaError_t _e = (expr);                                                           \
    if (_e != cudaSuccess) {                                                           \
      ::kpsb::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(_e)); \
      return KPSB_ECUDA;                                                               \
    }                                                                                  \
  } while (0)

#define KPSB_TRY(expr)                     \
  do {                                     \
    kpsb_status _s = (expr);               \
    if (_s != KPSB_OK) return _s;          \
  } while (0)

#define KPSB_CHECK_LAUNCH()     \
  do {                          \
    ::kpsb::count_launch();     \
    KPSB_TRY_CUDA(cudaGetLastError()); \
  } while (0)

#define KPSB_REQUIRE(cond, ...)            \
  do {                                     \
    if (!(cond)) {                         \
      ::kpsb::set_error(__VA_ARGS__);      \
      return KPSB_EINVAL;                  \
    }                                      \
  } while (0)

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// --------------------------------------------------------------------------------------
// Device helpers
// --------------------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (fixed order, deterministic).  All threads receive the result.
// `sh` must hold >= 32 elements.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T r = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (wid == 0) r = warp_sum(r);
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// Sum of `count` values p[0], p[stride], ... by the whole block in a fixed order: thread t
// adds entries t, t + blockDim.x, ... in turn, then block_sum combines the threads.  Used by
// the last block of a grid reduction, so the partials are read with __ldcg; many loads are in
// flight at once instead of one thread walking all partials.  All threads get the result.
__device__ __forceinline__ double block_sum_strided(const double* p, long long stride, int count,
                                                    double* sh) {
  double t = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) t += __ldcg(p + (long long)i * stride);
  return block_sum<double>(t, sh);
}

// The same by one warp (lanes stride, then the butterfly, whose lanes all end with the same
// bits: each level adds the same two values in either order).
__device__ __forceinline__ double warp_sum_strided(const double* p, long long stride, int count) {
  double t = 0.0;
  for (int i = threadIdx.x & 31; i < count; i += 32) t += __ldcg(p + (long long)i * stride);
  return warp_sum(t);
}

// "Last block" protocol of a deterministic grid reduction: every block writes its
// partial results, then calls this; exactly one block (the last to arrive) gets true and
// may read all partials (with __ldcg) in a fixed order.  The counter is reset by the
// last block so the next launch starts from zero.
__device__ __forceinline__ bool last_block_arrive(unsigned int* counter, unsigned int nblocks) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == nblocks - 1);
    if (s_last) *counter = 0u;  // no other block touches it again in this launch
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// Round to TF32 (10 explicit mantissa bits), to nearest with ties away from zero.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// The 1/2 forward-difference operators of the TV term on an n x n column-major image
// (L with a zero last row): Dx = (L (x) I) acts along columns, Dy = (I (x) L) along rows.
__device__ __forceinline__ double tv_dx(const double* X, int r, int c, int n) {  // (X L^T)(r,c)
  return c < n - 1 ? 0.5 * (X[r + (size_t)c * n] - X[r + (size_t)(c + 1) * n]) : 0.0;
}
__device__ __forceinline__ double tv_dy(const double* X, int r, int c, int n) {  // (L X)(r,c)
  return r < n - 1 ? 0.5 * (X[r + (size_t)c * n] - X[r + 1 + (size_t)c * n]) : 0.0;
}
__device__ __forceinline__ double tv_dxt(const double* Y, int r, int c, int n) {  // (Y L)(r,c)
  double v = c < n - 1 ? 0.5 * Y[r + (size_t)c * n] : 0.0;
  if (c >= 1) v -= 0.5 * Y[r + (size_t)(c - 1) * n];
  return v;
}
__device__ __forceinline__ double tv_dyt(const double* Y, int r, int c, int n) {  // (L^T Y)(r,c)
  double v = r < n - 1 ? 0.5 * Y[r + (size_t)c * n] : 0.0;
  if (r >= 1) v -= 0.5 * Y[r - 1 + (size_t)c * n];
  return v;
}

__device__ __forceinline__ int ext_index(int q, int n, int bc) {
  // Boundary extension: zero -> -1 for out-of-range; reflexive half-sample mirror.
  if (q >= 0 && q < n) return q;
  if (bc == KPSB_BC_ZERO) return -1;
  return q < 0 ? -1 - q : 2 * n - 1 - q;
}

}  // namespace kpsb

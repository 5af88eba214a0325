// Dense helpers of the TSVD phase: block dot products and updates of the (classical,
// two-pass) Gram-Schmidt reorthogonalisation, norms, Gram matrices, skinny products,
// the one-block FP64 Jacobi SVD and the Philox4x32-10 normal generator.
#include <math.h>

#include "jacobi.cuh"
#include "kpsb_internal.cuh"

namespace kpsb {

static constexpr int LA_THREADS = 256;

__device__ __forceinline__ bool gate_skip(const int* skip) { return skip && *skip; }

static int red_blocks(long long N, int per_thread) {
  long long b = (N + (long long)LA_THREADS * per_thread - 1) / ((long long)LA_THREADS * per_thread);
  return (int)std::max(1LL, std::min<long long>(b, RED_MAX_BLOCKS));
}

// The block helpers are templates on the basis element type: float for the single-
// precision TSVD, double for the FP64 one (reductions are FP64 in both).

// ---- h = S^T v --------------------------------------------------------------------------
// Each block owns a contiguous range of rows; for a chunk of DB columns every thread reads
// v[r] once and the DB basis entries of its rows (each read coalesced across the warp), then
// the chunk is reduced in a fixed order: a warp butterfly in the element type, the 8 warp
// totals in FP64 by DB threads, the blocks' FP64 partials by the last block.  One
// __syncthreads per chunk; FP64 work per block is O(DB * warps), not O(threads).
static constexpr int DB = 16;

template <typename T>
__global__ void __launch_bounds__(LA_THREADS) dot_block_kernel(
    const T* __restrict__ S, int ldS, int m, const T* __restrict__ v, long long N,
    double* __restrict__ part, unsigned int* __restrict__ counter, double* __restrict__ h,
    const int* skip) {
  if (gate_skip(skip)) return;
  __shared__ T wsum[LA_THREADS / 32][DB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long per = (N + gridDim.x - 1) / gridDim.x;
  const long long r_lo = (long long)blockIdx.x * per;
  const long long r_hi = r_lo + per < N ? r_lo + per : N;
  for (int c0 = 0; c0 < m; c0 += DB) {
    T acc[DB];
#pragma unroll
    for (int u = 0; u < DB; ++u) acc[u] = 0;
    for (long long r = r_lo + threadIdx.x; r < r_hi; r += LA_THREADS) {
      const T x = v[r];
      const T* sr = S + r + (size_t)c0 * ldS;
#pragma unroll
      for (int u = 0; u < DB; ++u)
        if (c0 + u < m) acc[u] = fma(sr[(size_t)u * ldS], x, acc[u]);
    }
#pragma unroll
    for (int u = 0; u < DB; ++u) {
      T t = acc[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      acc[u] = t;
    }
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < DB; ++u) wsum[warp][u] = acc[u];
    }
    __syncthreads();
    if (threadIdx.x < DB && c0 + (int)threadIdx.x < m) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < LA_THREADS / 32; ++w) t += (double)wsum[w][threadIdx.x];
      part[(size_t)blockIdx.x * m + c0 + threadIdx.x] = t;
    }
    __syncthreads();
  }
  if (!last_block_arrive(counter, gridDim.x)) return;
  for (int i = warp; i < m; i += LA_THREADS / 32) {  // one warp per column, fixed order
    const double t = warp_sum_strided(part + i, m, (int)gridDim.x);
    if (lane == 0) h[i] = t;
  }
}

template <typename T>
kpsb_status la_dot_block(const T* S, int ldS, int m, const T* v, long long N, double* h,
                         const RedScratch& red, const int* skip, cudaStream_t st) {
  if (m <= 0) return KPSB_OK;
  int nb = red_blocks(N, 4);
  dot_block_kernel<T><<<nb, LA_THREADS, 0, st>>>(S, ldS, m, v, N, red.part, red.counter, h, skip);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

// ---- v -= S h, optional ||v|| -------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(LA_THREADS) update_kernel(
    const T* __restrict__ S, int ldS, int m, const double* __restrict__ h, T* __restrict__ v,
    long long N, double* __restrict__ part, unsigned int* __restrict__ counter,
    double* __restrict__ norm_out, const int* skip) {
  if (gate_skip(skip)) return;
  __shared__ T hs[128];
  __shared__ double sh[32];
  for (int i = threadIdx.x; i < m; i += blockDim.x) hs[i] = (T)h[i];
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  T ss = 0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < N; r += stride) {
    T corr = 0;
    for (int i = 0; i < m; ++i) corr = fma(S[r + (size_t)i * ldS], hs[i], corr);
    T x = v[r] - corr;
    v[r] = x;
    ss = fma(x, x, ss);
  }
  if (!norm_out) return;
  double t = block_sum<double>((double)ss, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
  if (!last_block_arrive(counter, gridDim.x)) return;
  const double a = block_sum_strided(part, 1, (int)gridDim.x, sh);
  if (threadIdx.x == 0) *norm_out = sqrt(a);
}

template <typename T>
kpsb_status la_update(const T* S, int ldS, int m, const double* h, T* v, long long N,
                      double* norm_out, const RedScratch& red, const int* skip, cudaStream_t st) {
  int nb = red_blocks(N, 4);
  update_kernel<T><<<nb, LA_THREADS, 0, st>>>(S, ldS, m, h, v, N, red.part, red.counter, norm_out, skip);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

template <typename T>
kpsb_status la_norm(const T* v, long long N, double* norm_out, const RedScratch& red,
                    const int* skip, cudaStream_t st) {
  return la_update<T>(nullptr, 0, 0, nullptr, const_cast<T*>(v), N, norm_out, red, skip, st);
}

template <typename T>
__global__ void scale_inv_kernel(T* __restrict__ v, long long N, const double* __restrict__ nrm,
                                 const int* skip) {
  if (gate_skip(skip)) return;
  double d = *nrm;
  T s = d > 0.0 ? (T)(1.0 / d) : (T)0;  // zero norm: the vector is cleared
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < N;
       r += (long long)gridDim.x * blockDim.x)
    v[r] *= s;
}

template <typename T>
kpsb_status la_scale_inv(T* v, long long N, const double* norm, const int* skip, cudaStream_t st) {
  int nb = (int)std::min<long long>((N + 1023) / 1024, 1216);
  scale_inv_kernel<T><<<nb, LA_THREADS, 0, st>>>(v, N, norm, skip);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

// ---- G = Y^T Y (FP64) ----------------------------------------------------------------------
// Blocks take contiguous ranges of 64-row tiles; a tile is staged in shared memory already
// widened to FP64 (one conversion per element, not per product) and each thread forms its
// pairs i <= j of the upper triangle (m (m + 1) / 2 <= 2080 pairs, at most 9 per thread).
// Partials per block, summed in a fixed order by the last block, which mirrors the triangle.
static constexpr int GR_ROWS = 64;
static constexpr int GR_PAIRS = 9;  // ceil(64 * 65 / 2 / 256)

template <typename T>
__global__ void __launch_bounds__(LA_THREADS) gram_kernel(const T* __restrict__ Y, int ldy,
                                                         long long N, int m,
                                                         double* __restrict__ part,
                                                         unsigned int* __restrict__ counter,
                                                         double* __restrict__ G) {
  __shared__ double ch[GR_ROWS][65];
  const int npair = m * (m + 1) / 2;
  int pi[GR_PAIRS], pj[GR_PAIRS];
#pragma unroll
  for (int u = 0; u < GR_PAIRS; ++u) {  // pair p -> (i, j), i <= j, column j of the triangle
    int p = threadIdx.x + u * LA_THREADS, j = 0;
    if (p < npair) {
      while ((j + 1) * (j + 2) / 2 <= p) ++j;
      pi[u] = p - j * (j + 1) / 2;
      pj[u] = j;
    } else {
      pi[u] = pj[u] = 0;
    }
  }
  double acc[GR_PAIRS];
#pragma unroll
  for (int u = 0; u < GR_PAIRS; ++u) acc[u] = 0.0;
  const long long tiles = (N + GR_ROWS - 1) / GR_ROWS;
  const long long per = (tiles + gridDim.x - 1) / gridDim.x;
  const long long t_lo = (long long)blockIdx.x * per, t_hi = t_lo + per < tiles ? t_lo + per : tiles;
  for (long long tb = t_lo; tb < t_hi; ++tb) {
    const long long rb = tb * GR_ROWS;
    __syncthreads();
    for (int e = threadIdx.x; e < GR_ROWS * m; e += blockDim.x) {
      int rr = e % GR_ROWS, c = e / GR_ROWS;
      long long r = rb + rr;
      ch[rr][c] = r < N ? (double)Y[r + (size_t)c * ldy] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < GR_PAIRS; ++u) {
      if (threadIdx.x + u * LA_THREADS < npair) {
        const int i = pi[u], j = pj[u];
        double a = 0.0;
#pragma unroll 8
        for (int rr = 0; rr < GR_ROWS; ++rr) a = fma(ch[rr][i], ch[rr][j], a);
        acc[u] += a;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < GR_PAIRS; ++u) {
    int p = threadIdx.x + u * LA_THREADS;
    if (p < npair) part[(size_t)blockIdx.x * npair + p] = acc[u];
  }
  if (!last_block_arrive(counter, gridDim.x)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int p = warp; p < npair; p += LA_THREADS / 32) {  // one warp per pair, fixed order
    const double a = warp_sum_strided(part + p, npair, (int)gridDim.x);
    if (lane == 0) {
      int j = 0;
      while ((j + 1) * (j + 2) / 2 <= p) ++j;
      const int i = p - j * (j + 1) / 2;
      G[i + (size_t)j * m] = a;  // column-major, both triangles
      G[j + (size_t)i * m] = a;
    }
  }
}

template <typename T>
kpsb_status la_gram(const T* Y, int ldy, long long N, int m, double* G, const RedScratch& red,
                    cudaStream_t st) {
  KPSB_REQUIRE(m >= 1 && m <= 64, "gram width %d outside [1,64]", m);
  int nb = (int)std::max(1LL, std::min<long long>((N + GR_ROWS - 1) / GR_ROWS, 2 * 152));
  gram_kernel<T><<<nb, LA_THREADS, 0, st>>>(Y, ldy, N, m, red.part, red.counter, G);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

// ---- Out = Y T --------------------------------------------------------------------------------
template <typename TY, typename TO>
__global__ void __launch_bounds__(LA_THREADS) matmul_small_kernel(
    const TY* __restrict__ Y, int ldy, long long N, int m, const double* __restrict__ T, int ldt,
    int kk, TO* __restrict__ Out, int ldo) {
  __shared__ TY Ts[64 * 64];
  for (int e = threadIdx.x; e < m * kk; e += blockDim.x) {
    int i = e % m, j = e / m;
    Ts[i + j * 64] = (TY)T[i + (size_t)j * ldt];
  }
  __syncthreads();
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < N;
       r += (long long)gridDim.x * blockDim.x) {
    for (int j0 = 0; j0 < kk; j0 += 16) {
      TY acc[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) acc[u] = 0;
      for (int i = 0; i < m; ++i) {
        TY y = Y[r + (size_t)i * ldy];
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] = fma(y, Ts[i + (j0 + u) * 64], acc[u]);
      }
#pragma unroll
      for (int u = 0; u < 16; ++u)
        if (j0 + u < kk) Out[r + (size_t)(j0 + u) * ldo] = (TO)acc[u];
    }
  }
}

template <typename TY, typename TO>
kpsb_status la_matmul_small(const TY* Y, int ldy, long long N, int m, const double* T, int ldt,
                            int kk, TO* Out, int ldo, cudaStream_t st) {
  KPSB_REQUIRE(m >= 1 && m <= 64 && kk >= 1 && kk <= 64, "small matmul %dx%d outside 64", m, kk);
  int nb = (int)std::min<long long>((N + LA_THREADS - 1) / LA_THREADS, 152 * 8);
  matmul_small_kernel<TY, TO><<<nb, LA_THREADS, 0, st>>>(Y, ldy, N, m, T, ldt, kk, Out, ldo);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

// element-type conversion (start vectors given in FP32 to the FP64 TSVD)
template <typename TO, typename TI>
__global__ void convert_kernel(const TI* __restrict__ in, TO* __restrict__ out, long long N) {
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < N;
       r += (long long)gridDim.x * blockDim.x)
    out[r] = (TO)in[r];
}

template <typename TO, typename TI>
kpsb_status la_convert(const TI* in, TO* out, long long N, cudaStream_t st) {
  int nb = (int)std::min<long long>((N + 255) / 256, 152 * 8);
  convert_kernel<TO, TI><<<std::max(1, nb), 256, 0, st>>>(in, out, N);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

template kpsb_status la_dot_block<float>(const float*, int, int, const float*, long long, double*, const RedScratch&, const int*, cudaStream_t);
template kpsb_status la_dot_block<double>(const double*, int, int, const double*, long long, double*, const RedScratch&, const int*, cudaStream_t);
template kpsb_status la_update<float>(const float*, int, int, const double*, float*, long long, double*, const RedScratch&, const int*, cudaStream_t);
template kpsb_status la_update<double>(const double*, int, int, const double*, double*, long long, double*, const RedScratch&, const int*, cudaStream_t);
template kpsb_status la_norm<float>(const float*, long long, double*, const RedScratch&, const int*, cudaStream_t);
template kpsb_status la_norm<double>(const double*, long long, double*, const RedScratch&, const int*, cudaStream_t);
template kpsb_status la_scale_inv<float>(float*, long long, const double*, const int*, cudaStream_t);
template kpsb_status la_scale_inv<double>(double*, long long, const double*, const int*, cudaStream_t);
template kpsb_status la_gram<float>(const float*, int, long long, int, double*, const RedScratch&, cudaStream_t);
template kpsb_status la_gram<double>(const double*, int, long long, int, double*, const RedScratch&, cudaStream_t);
template kpsb_status la_matmul_small<float, float>(const float*, int, long long, int, const double*, int, int, float*, int, cudaStream_t);
template kpsb_status la_matmul_small<double, double>(const double*, int, long long, int, const double*, int, int, double*, int, cudaStream_t);
template kpsb_status la_matmul_small<double, float>(const double*, int, long long, int, const double*, int, int, float*, int, cudaStream_t);
template kpsb_status la_convert<double, float>(const float*, double*, long long, cudaStream_t);

// ---- one-sided Jacobi SVD (Hestenes) in one thread block: jacobi.cuh ----------------------
__global__ void __launch_bounds__(1024) jacobi_svd_kernel(const double* __restrict__ A, int lda,
                                                        int m, int nc, double* __restrict__ U,
                                                        double* __restrict__ S,
                                                        double* __restrict__ V,
                                                        int* __restrict__ sweeps_out,
                                                        int max_sweeps) {
  extern __shared__ double smem[];
  jacobi_svd_block(A, lda, m, nc, U, S, V, sweeps_out, max_sweeps, smem);
}

kpsb_status la_small_svd(const double* A, int lda, int m, int nc, double* U, double* S, double* V,
                         int* sweeps, cudaStream_t st) {
  KPSB_REQUIRE(nc >= 1 && nc <= 64 && m >= nc && m <= 128, "small SVD %dx%d outside limits", m, nc);
  size_t sm = (size_t)(m * nc + nc * nc) * sizeof(double);
  KPSB_TRY_CUDA(cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (128 * 64 + 64 * 64) * (int)sizeof(double)));
  // JL lanes per column pair, every rotation of a round at once
  const int pairs = (nc + (nc & 1)) / 2;
  const int warps = std::max(1, (pairs + 32 / JL - 1) / (32 / JL));
  jacobi_svd_kernel<<<1, 32 * warps, sm, st>>>(A, lda, m, nc, U, S, V, sweeps, 60);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) + Box-Muller ---------------------------
__device__ __forceinline__ void philox_round(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3,
                                             uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  uint32_t hi0 = __umulhi(M0, x0), lo0 = M0 * x0;
  uint32_t hi1 = __umulhi(M1, x2), lo1 = M1 * x2;
  uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
  x0 = y0; x1 = y1; x2 = y2; x3 = y3;
}

template <typename T>
__global__ void randn_kernel(T* __restrict__ out, long long count, uint32_t key0, uint32_t key1) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g * 4 < count;
       g += (long long)gridDim.x * blockDim.x) {
    uint32_t x0 = (uint32_t)g, x1 = (uint32_t)(g >> 32), x2 = 0u, x3 = 0u;
    uint32_t k0 = key0, k1 = key1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      philox_round(x0, x1, x2, x3, k0, k1);
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t xs[4] = {x0, x1, x2, x3};
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
      long long i0 = g * 4 + 2 * pr;
      if (sizeof(T) == sizeof(float)) {
        // single-precision bases: the transform in FP32 (GB300's FP64 pipe is narrow)
        float u1 = ((float)(xs[2 * pr] >> 8) + 1.0f) * 5.9604644775390625e-08f;  // (0, 1], 24 bits
        float u2 = (float)(xs[2 * pr + 1] >> 8) * 5.9604644775390625e-08f;        // [0, 1)
        float rad = sqrtf(-2.0f * logf(u1)), sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        if (i0 < count) out[i0] = (T)(rad * cs);
        if (i0 + 1 < count) out[i0 + 1] = (T)(rad * sn);
      } else {
        double u1 = ((double)xs[2 * pr] + 1.0) * 2.3283064365386963e-10;  // (0, 1]
        double u2 = (double)xs[2 * pr + 1] * 2.3283064365386963e-10;       // [0, 1)
        double rad = sqrt(-2.0 * log(u1));
        double th = 6.283185307179586 * u2;
        if (i0 < count) out[i0] = (T)(rad * cos(th));
        if (i0 + 1 < count) out[i0 + 1] = (T)(rad * sin(th));
      }
    }
  }
}

template <typename T>
kpsb_status la_randn(T* out, long long count, unsigned long long seed, cudaStream_t st) {
  int nb = (int)std::min<long long>((count / 4 + 255) / 256 + 1, 152 * 8);
  randn_kernel<T><<<nb, 256, 0, st>>>(out, count, (uint32_t)seed, (uint32_t)(seed >> 32));
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}
template kpsb_status la_randn<float>(float*, long long, unsigned long long, cudaStream_t);
template kpsb_status la_randn<double>(double*, long long, unsigned long long, cudaStream_t);

}  // namespace kpsb

// ---- C ABI: small SVD (host pointers, synchronous) ---------------------------------------------
using namespace kpsb;
extern "C" kpsb_status kpsb_small_svd(int m, int nc, const double* A, double* U, double* S,
                                      double* V, int* sweeps) {
  clear_error();
  KPSB_REQUIRE(A && U && S && V, "null pointer");
  KPSB_REQUIRE(nc >= 1 && nc <= 64 && m >= nc && m <= 128, "small SVD %dx%d outside limits", m, nc);
  double* d = nullptr;
  size_t tot = (size_t)(2 * m * nc + nc + nc * nc) * sizeof(double) + sizeof(int);
  KPSB_TRY_CUDA(cudaMalloc(&d, tot));
  double *dA = d, *dU = dA + m * nc, *dS = dU + m * nc, *dV = dS + nc;
  int* dsw = (int*)(dV + nc * nc);
  kpsb_status s = KPSB_OK;
  cudaError_t e = cudaMemcpy(dA, A, sizeof(double) * m * nc, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    s = la_small_svd(dA, m, m, nc, dU, dS, dV, dsw, 0);
    if (s == KPSB_OK) e = cudaDeviceSynchronize();
  }
  if (e == cudaSuccess && s == KPSB_OK) {
    cudaMemcpy(U, dU, sizeof(double) * m * nc, cudaMemcpyDeviceToHost);
    cudaMemcpy(S, dS, sizeof(double) * nc, cudaMemcpyDeviceToHost);
    cudaMemcpy(V, dV, sizeof(double) * nc * nc, cudaMemcpyDeviceToHost);
    int sw = 0;
    e = cudaMemcpy(&sw, dsw, sizeof(int), cudaMemcpyDeviceToHost);
    if (sweeps) *sweeps = sw;
  }
  cudaFree(d);
  if (e != cudaSuccess) {
    set_error("small SVD: %s", cudaGetErrorString(e));
    return KPSB_ECUDA;
  }
  return s;
}

// Kronecker-sum operator apply (Sec. 4.2, eq. (4.3)) on CUDA cores, batched over problems:
//   forward   Y  = sum_i sigma_i Ay_i X Ax_i^T
//   transpose X' = sum_i sigma_i Ay_i^T Y Ax_i
// as two GEMM stages per problem and term, Z_i = sigma_i X op(Ax_i) and W_i = op(Ay_i) Z_i,
// then Y = sum_i W_i in term order (deterministic).  FP64 mode accumulates in FP64 (the plain
// path); FP32 mode rounds X to FP32 and accumulates in FP32.
#include "kpsb_internal.cuh"

namespace kpsb {

// 32 x 32 output tiles, K slices of 16, 256 threads with 2 x 2 outputs each: small tiles and
// one CTA per (tile, term) in both stages keep a single n = 128 problem on ~16 k CTAs.
static constexpr int GT = 32, GB_K = 16, GB_T = 256;

// Work actually performed by the applies of this file (as in the tensor-core file):
// [0] sum of k n^3 over active problems, [1] active problem-applies.
__device__ unsigned long long g_simt_work[2] = {0, 0};

// Load a GB_K x GT operand tile into smem s[kk][mm] from src(mm, kk) = base[mm*sm + kk*sk].
template <typename TA, typename TS>
__device__ __forceinline__ void load_tile(TS (*s)[GT + 1], const TA* __restrict__ base, int sm, int sk,
                                          int mlim, int klim) {
#pragma unroll
  for (int u = 0; u < (GT * GB_K) / GB_T; ++u) {
    const int e = threadIdx.x + u * GB_T;
    int mm, kk;
    if (sm == 1) {  // contiguous along m
      mm = e % GT;
      kk = e / GT;
    } else {        // contiguous along k
      kk = e % GB_K;
      mm = e / GB_K;
    }
    s[kk][mm] = (mm < mlim && kk < klim) ? (TS)base[(size_t)mm * sm + (size_t)kk * sk] : (TS)0;
  }
}

// acc[x][y] += sum_kk As[kk][tx + 16x] Bs[kk][ty + 16y]
template <typename TAcc>
__device__ __forceinline__ void mma_tile(const TAcc (*As)[GT + 1], const TAcc (*Bs)[GT + 1], TAcc acc[2][2],
                                         int tx, int ty) {
#pragma unroll
  for (int kk = 0; kk < GB_K; ++kk) {
    const TAcc a0 = As[kk][tx], a1 = As[kk][tx + 16], b0 = Bs[kk][ty], b1 = Bs[kk][ty + 16];
    acc[0][0] = fma(a0, b0, acc[0][0]);
    acc[0][1] = fma(a0, b1, acc[0][1]);
    acc[1][0] = fma(a1, b0, acc[1][0]);
    acc[1][1] = fma(a1, b1, acc[1][1]);
  }
}

// Stage 1: Z_i(r, j) = sigma_i sum_l X(r, l) B(l, j), with B(l, j) = Ax_i(j, l) (forward) or
// Ax_i(l, j) (transpose).  grid = (tiles, kmax, njobs).
template <typename TAcc, typename TZ>
__global__ void __launch_bounds__(GB_T) kp_stage1_kernel(const KPJob* __restrict__ jobs, int transpose) {
  const KPJob J = jobs[blockIdx.z];
  const int i = blockIdx.y;
  if (i >= J.k || (J.active && !*J.active)) return;
  const int n = J.n;
  const int tiles_m = (n + GT - 1) / GT;
  const int m0 = (blockIdx.x % tiles_m) * GT, n0 = (blockIdx.x / tiles_m) * GT;
  if (n0 >= n) return;
  __shared__ TAcc As[GB_K][GT + 1];
  __shared__ TAcc Bs[GB_K][GT + 1];
  const float* Ax = J.Ax + (size_t)i * n * n;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  TAcc acc[2][2] = {{0, 0}, {0, 0}};
  for (int k0 = 0; k0 < n; k0 += GB_K) {
    load_tile<double, TAcc>(As, J.X + m0 + (size_t)k0 * n, 1, n, n - m0, n - k0);  // X(r, l)
    if (!transpose)
      load_tile<float, TAcc>(Bs, Ax + n0 + (size_t)k0 * n, 1, n, n - n0, n - k0);  // Ax(j, l)
    else
      load_tile<float, TAcc>(Bs, Ax + (size_t)n0 * n + k0, n, 1, n - n0, n - k0);  // Ax(l, j)
    __syncthreads();
    mma_tile<TAcc>(As, Bs, acc, tx, ty);
    __syncthreads();
  }
  const TAcc sg = (TAcc)J.sigma[i];
  TZ* Z = (TZ*)J.Z + (size_t)i * n * n;
#pragma unroll
  for (int y = 0; y < 2; ++y) {
    const int c = n0 + ty + 16 * y;
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      const int r = m0 + tx + 16 * x;
      if (r < n && c < n) Z[r + (size_t)c * n] = (TZ)(sg * acc[x][y]);
    }
  }
}

// Stage 2, one term per CTA: W_i(r, c) = sum_l A_i(r, l) Z_i(l, c), A_i(r, l) = Ay_i(r, l)
// (forward) or Ay_i(l, r) (transpose), into the partial buffer after Z.  grid = (tiles,
// kmax, njobs).
template <typename TAcc, typename TZ>
__global__ void __launch_bounds__(GB_T) kp_stage2_kernel(const KPJob* __restrict__ jobs, int transpose) {
  const KPJob J = jobs[blockIdx.z];
  const int i = blockIdx.y;
  if (i >= J.k || (J.active && !*J.active)) return;
  const int n = J.n;
  if (blockIdx.x == 0 && i == 0 && threadIdx.x == 0) {
    atomicAdd(&g_simt_work[0], (unsigned long long)J.k * n * n * n);
    atomicAdd(&g_simt_work[1], 1ull);
  }
  const int tiles_m = (n + GT - 1) / GT;
  const int m0 = (blockIdx.x % tiles_m) * GT, n0 = (blockIdx.x / tiles_m) * GT;
  if (n0 >= n) return;
  __shared__ TAcc As[GB_K][GT + 1];
  __shared__ TAcc Bs[GB_K][GT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const size_t nn = (size_t)n * n;
  const float* Ay = J.Ay + (size_t)i * nn;
  const TZ* Z = (const TZ*)J.Z + (size_t)i * nn;
  TAcc acc[2][2] = {{0, 0}, {0, 0}};
  for (int k0 = 0; k0 < n; k0 += GB_K) {
    if (!transpose)
      load_tile<float, TAcc>(As, Ay + m0 + (size_t)k0 * n, 1, n, n - m0, n - k0);
    else
      load_tile<float, TAcc>(As, Ay + (size_t)m0 * n + k0, n, 1, n - m0, n - k0);
    load_tile<TZ, TAcc>(Bs, Z + (size_t)n0 * n + k0, n, 1, n - n0, n - k0);  // Z(l, c)
    __syncthreads();
    mma_tile<TAcc>(As, Bs, acc, tx, ty);
    __syncthreads();
  }
  TZ* W = (TZ*)J.Z + (size_t)J.k * nn + (size_t)i * nn;
#pragma unroll
  for (int y = 0; y < 2; ++y) {
    const int c = n0 + ty + 16 * y;
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      const int r = m0 + tx + 16 * x;
      if (r < n && c < n) W[r + (size_t)c * n] = (TZ)acc[x][y];
    }
  }
}

// Y = sum_i W_i in term order.  grid = (blocks, njobs).
template <typename TAcc, typename TZ>
__global__ void kp_sum_terms_kernel(const KPJob* __restrict__ jobs) {
  const KPJob J = jobs[blockIdx.y];
  if (J.active && !*J.active) return;
  const size_t nn = (size_t)J.n * J.n;
  const TZ* W = (const TZ*)J.Z + (size_t)J.k * nn;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn; e += (size_t)gridDim.x * blockDim.x) {
    TAcc s = 0;
    for (int i = 0; i < J.k; ++i) s += (TAcc)W[(size_t)i * nn + e];
    J.Y[e] = (double)s;
  }
}

kpsb_status simt_work(unsigned long long* out, bool reset) {
  if (reset) {
    const unsigned long long z[2] = {0, 0};
    KPSB_TRY_CUDA(cudaMemcpyToSymbol(g_simt_work, z, sizeof(z)));
  }
  if (out) KPSB_TRY_CUDA(cudaMemcpyFromSymbol(out, g_simt_work, 2 * sizeof(unsigned long long)));
  return KPSB_OK;
}

// Z (k n^2) and the per-term partials W (k n^2), in the accumulation type.
size_t kp_z_bytes(int n, int k, int prec) {
  size_t el = prec == KPSB_P_FP64 ? sizeof(double) : sizeof(float);
  return 2 * el * (size_t)n * n * k;
}

template <typename TAcc>
static kpsb_status launch_simt(const KPJob* jobs_d, int njobs, int n, int kmax, int transpose, cudaStream_t st) {
  const int tiles = ((n + GT - 1) / GT) * ((n + GT - 1) / GT);
  dim3 g12(tiles, kmax, njobs);
  kp_stage1_kernel<TAcc, TAcc><<<g12, GB_T, 0, st>>>(jobs_d, transpose);
  KPSB_CHECK_LAUNCH();
  kp_stage2_kernel<TAcc, TAcc><<<g12, GB_T, 0, st>>>(jobs_d, transpose);
  KPSB_CHECK_LAUNCH();
  const size_t nn = (size_t)n * n;
  dim3 g3((unsigned)std::min<size_t>((nn + 255) / 256, 1024), njobs);
  kp_sum_terms_kernel<TAcc, TAcc><<<g3, 256, 0, st>>>(jobs_d);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

kpsb_status kp_apply_batch(const KPJob* jobs_d, int njobs, int n, int kmax, int transpose, int prec,
                           cudaStream_t st) {
  if (njobs <= 0 || kmax <= 0) return KPSB_OK;
  if (prec == KPSB_P_FP64) return launch_simt<double>(jobs_d, njobs, n, kmax, transpose, st);
  if (prec == KPSB_P_FP32) return launch_simt<float>(jobs_d, njobs, n, kmax, transpose, st);
  set_error("precision %d is not a CUDA-core mode", prec);
  return KPSB_EINVAL;
}

}  // namespace kpsb

using namespace kpsb;

extern "C" kpsb_status kp_apply_dev(kpsb_kp_t kp, const double* X, double* Y, int transpose, int prec,
                                    void* stream) {
  clear_error();
  KPSB_REQUIRE(kp && X && Y && X != Y, "null or aliased pointer");
  KPSB_REQUIRE(prec_valid(prec), "unknown precision %d", prec);
  cudaStream_t st = (cudaStream_t)stream;
  const int n = kp->n, k = kp->k;
  if (kp->A_dense) {  // explicit operator: FP64 products
    KPSB_REQUIRE(prec == KPSB_P_FP64, "an explicit-operator handle applies in FP64 only");
    double* part = nullptr;
    KPSB_TRY_CUDA(cudaMallocAsync((void**)&part, sizeof(double) * dense_partials(n) + 256, st));
    KPJob J{};
    J.n = n;
    J.X = X;
    J.Y = Y;
    J.A = kp->A_dense;
    J.Z = (char*)part + 256;
    KPJob* Jd = (KPJob*)part;
    cudaError_t e = cudaMemcpyAsync(Jd, &J, sizeof(KPJob), cudaMemcpyHostToDevice, st);
    kpsb_status s = KPSB_OK;
    if (e == cudaSuccess) s = dense_apply_batch(Jd, 1, n, transpose, st);
    cudaError_t e2 = cudaStreamSynchronize(st);  // the descriptor copy is from the host stack
    cudaFreeAsync(part, st);
    if (e != cudaSuccess || (s == KPSB_OK && e2 != cudaSuccess)) {
      set_error("kp_apply_dev (explicit A): %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
      return KPSB_ECUDA;
    }
    return s;
  }
  const bool tc = tc_supported(kp->n, prec);
  if (prec_is_tc(prec) && !tc) prec = KPSB_P_FP32;  // sizes below the tensor-core tiles
  size_t zb = tc ? 0 : kp_z_bytes(n, k, prec);
  char* buf = nullptr;
  KPSB_TRY_CUDA(cudaMallocAsync((void**)&buf, zb + 256, st));
  KPJob J{};
  J.Ax = kp->Ax;
  J.Ay = kp->Ay;
  J.sigma = kp->sigma_d;
  J.n = n;
  J.k = k;
  J.X = X;
  J.Y = Y;
  J.Z = buf + 256;
  J.active = nullptr;
  KPJob* Jd = (KPJob*)buf;
  kpsb_status s = KPSB_OK;
  cudaError_t e = cudaMemcpyAsync(Jd, &J, sizeof(KPJob), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    set_error("kp_apply_dev: %s", cudaGetErrorString(e));
    s = KPSB_ECUDA;
  } else {
    int slot = gemm_timer_begin(st);
    if (tc) {
      kpsb_kp* kps[1] = {kp};
      s = tc_apply_batch(kps, Jd, &J, 1, n, k, transpose, prec, st);
    } else {
      s = kp_apply_batch(Jd, 1, n, k, transpose, prec, st);
    }
    gemm_timer_end(slot, st, 4.0 * k * (double)n * n * n, tc ? 1 : 3);
  }
  // the descriptor copy is from host stack memory: wait for it before returning
  cudaError_t e2 = cudaStreamSynchronize(st);
  cudaFreeAsync(buf, st);
  if (s == KPSB_OK && e2 != cudaSuccess) {
    set_error("kp_apply_dev: %s", cudaGetErrorString(e2));
    s = KPSB_ECUDA;
  }
  return s;
}

extern "C" kpsb_status kp_apply(kpsb_kp_t kp, const double* X, double* Y, int transpose, int prec) {
  clear_error();
  KPSB_REQUIRE(kp && X && Y, "null pointer");
  const size_t bytes = sizeof(double) * (size_t)kp->n * kp->n;
  double* d = nullptr;
  KPSB_TRY_CUDA(cudaMalloc(&d, 2 * bytes));
  kpsb_status s = KPSB_OK;
  cudaError_t e = cudaMemcpy(d, X, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    s = kp_apply_dev(kp, d, d + bytes / sizeof(double), transpose, prec, nullptr);
    if (s == KPSB_OK) e = cudaMemcpy(Y, d + bytes / sizeof(double), bytes, cudaMemcpyDeviceToHost);
  }
  cudaFree(d);
  if (e != cudaSuccess) {
    set_error("kp_apply: %s", cudaGetErrorString(e));
    return KPSB_ECUDA;
  }
  return s;
}

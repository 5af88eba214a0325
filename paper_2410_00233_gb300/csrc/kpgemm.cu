// Kronecker-sum operator apply (Sec. 4.2, eq. (4.3)) on CUDA cores, batched over problems:
//   forward   Y  = sum_i sigma_i Ay_i X Ax_i^T
//   transpose X' = sum_i sigma_i Ay_i^T Y Ax_i
// as two GEMM stages per problem: Z_i = sigma_i X op(Ax_i) (one tile grid per term), then
// Y = sum_i op(Ay_i) Z_i (K dimension = k*n).  FP64 mode accumulates in FP64 (the plain
// path); FP32 mode rounds X to FP32 and accumulates in FP32.
#include "kpsb_internal.cuh"

namespace kpsb {

static constexpr int GB_M = 64, GB_N = 64, GB_K = 16, GB_T = 256;

// Work actually performed by the applies of this file (as in the tensor-core file):
// [0] sum of k n^3 over active problems, [1] active problem-applies.
__device__ unsigned long long g_simt_work[2] = {0, 0};

template <typename T>
struct TileOps;

// Load a GB_K x 64 operand tile into smem s[kk][mm] from src(mm, kk) = base[mm*sm + kk*sk].
template <typename TA, typename TS>
__device__ __forceinline__ void load_tile(TS (*s)[GB_M + 1], const TA* __restrict__ base, int sm,
                                          int sk, int mlim, int klim) {
  if (sm == 1) {
#pragma unroll
    for (int u = 0; u < (GB_M * GB_K) / GB_T; ++u) {
      int e = threadIdx.x + u * GB_T;
      int mm = e % GB_M, kk = e / GB_M;
      s[kk][mm] = (mm < mlim && kk < klim) ? (TS)base[(size_t)mm + (size_t)kk * sk] : (TS)0;
    }
  } else {
#pragma unroll
    for (int u = 0; u < (GB_M * GB_K) / GB_T; ++u) {
      int e = threadIdx.x + u * GB_T;
      int kk = e % GB_K, mm = e / GB_K;
      s[kk][mm] = (mm < mlim && kk < klim) ? (TS)base[(size_t)mm * sm + (size_t)kk * sk] : (TS)0;
    }
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
  const int tiles_m = (n + GB_M - 1) / GB_M;
  const int m0 = (blockIdx.x % tiles_m) * GB_M, n0 = (blockIdx.x / tiles_m) * GB_N;
  if (n0 >= n) return;
  __shared__ TAcc As[GB_K][GB_M + 1];
  __shared__ TAcc Bs[GB_K][GB_N + 1];
  const float* Ax = J.Ax + (size_t)i * n * n;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  TAcc acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
  for (int k0 = 0; k0 < n; k0 += GB_K) {
    // A(r, l) = X[r + l n]
    load_tile<double, TAcc>(As, J.X + m0 + (size_t)k0 * n, 1, n, n - m0, n - k0);
    // B(l, j): forward Ax[j + l n] (j stride 1), transpose Ax[l + j n] (l stride 1)
    if (!transpose)
      load_tile<float, TAcc>(Bs, Ax + n0 + (size_t)k0 * n, 1, n, n - n0, n - k0);
    else
      load_tile<float, TAcc>(Bs, Ax + (size_t)n0 * n + k0, n, 1, n - n0, n - k0);
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GB_K; ++kk) {
      TAcc a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = As[kk][tx + 16 * u];
#pragma unroll
      for (int u = 0; u < 4; ++u) b[u] = Bs[kk][ty + 16 * u];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
  const TAcc sg = (TAcc)J.sigma[i];
  TZ* Z = (TZ*)J.Z + (size_t)i * n * n;
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    int c = n0 + ty + 16 * y;
    if (c >= n) continue;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      int r = m0 + tx + 16 * x;
      if (r < n) Z[r + (size_t)c * n] = (TZ)(sg * acc[x][y]);
    }
  }
}

// Stage 2: Y(r, c) = sum_i sum_l A_i(r, l) Z_i(l, c), A_i(r, l) = Ay_i(r, l) (forward) or
// Ay_i(l, r) (transpose).  grid = (tiles, 1, njobs).
template <typename TAcc, typename TZ>
__global__ void __launch_bounds__(GB_T) kp_stage2_kernel(const KPJob* __restrict__ jobs, int transpose) {
  const KPJob J = jobs[blockIdx.z];
  if (J.active && !*J.active) return;
  const int n = J.n;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAdd(&g_simt_work[0], (unsigned long long)J.k * n * n * n);
    atomicAdd(&g_simt_work[1], 1ull);
  }
  const int tiles_m = (n + GB_M - 1) / GB_M;
  const int m0 = (blockIdx.x % tiles_m) * GB_M, n0 = (blockIdx.x / tiles_m) * GB_N;
  if (n0 >= n) return;
  __shared__ TAcc As[GB_K][GB_M + 1];
  __shared__ TAcc Bs[GB_K][GB_N + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  TAcc acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
  for (int i = 0; i < J.k; ++i) {
    const float* Ay = J.Ay + (size_t)i * n * n;
    const TZ* Z = (const TZ*)J.Z + (size_t)i * n * n;
    for (int k0 = 0; k0 < n; k0 += GB_K) {
      if (!transpose)
        load_tile<float, TAcc>(As, Ay + m0 + (size_t)k0 * n, 1, n, n - m0, n - k0);
      else
        load_tile<float, TAcc>(As, Ay + (size_t)m0 * n + k0, n, 1, n - m0, n - k0);
      // B(l, c) = Z[l + c n]
      load_tile<TZ, TAcc>(Bs, Z + (size_t)n0 * n + k0, n, 1, n - n0, n - k0);
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < GB_K; ++kk) {
        TAcc a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = As[kk][tx + 16 * u];
#pragma unroll
        for (int u = 0; u < 4; ++u) b[u] = Bs[kk][ty + 16 * u];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    int c = n0 + ty + 16 * y;
    if (c >= n) continue;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      int r = m0 + tx + 16 * x;
      if (r < n) J.Y[r + (size_t)c * n] = (double)acc[x][y];
    }
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

size_t kp_z_bytes(int n, int k, int prec) {
  size_t el = prec == KPSB_P_FP64 ? sizeof(double) : sizeof(float);
  return el * (size_t)n * n * k;
}

kpsb_status kp_apply_batch(const KPJob* jobs_d, int njobs, int n, int kmax, int transpose, int prec,
                           cudaStream_t st) {
  if (njobs <= 0 || kmax <= 0) return KPSB_OK;
  const int tiles = ((n + GB_M - 1) / GB_M) * ((n + GB_N - 1) / GB_N);
  dim3 g1(tiles, kmax, njobs), g2(tiles, 1, njobs);
  if (prec == KPSB_P_FP64) {
    kp_stage1_kernel<double, double><<<g1, GB_T, 0, st>>>(jobs_d, transpose);
    KPSB_CHECK_LAUNCH();
    kp_stage2_kernel<double, double><<<g2, GB_T, 0, st>>>(jobs_d, transpose);
  } else if (prec == KPSB_P_FP32) {
    kp_stage1_kernel<float, float><<<g1, GB_T, 0, st>>>(jobs_d, transpose);
    KPSB_CHECK_LAUNCH();
    kp_stage2_kernel<float, float><<<g2, GB_T, 0, st>>>(jobs_d, transpose);
  } else {
    set_error("precision %d is not a CUDA-core mode", prec);
    return KPSB_EINVAL;
  }
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

}  // namespace kpsb

using namespace kpsb;

extern "C" kpsb_status kp_apply_dev(kpsb_kp_t kp, const double* X, double* Y, int transpose, int prec,
                                    void* stream) {
  clear_error();
  KPSB_REQUIRE(kp && X && Y && X != Y, "null or aliased pointer");
  KPSB_REQUIRE(prec >= KPSB_P_FP64 && prec <= KPSB_P_TF32X2, "unknown precision %d", prec);
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
  if ((prec == KPSB_P_TF32X3 || prec == KPSB_P_TF32X2) && !tc) prec = KPSB_P_FP32;  // untiled sizes
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
    gemm_timer_end(slot, st, 4.0 * k * (double)n * n * n, tc ? 1 : 2);
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

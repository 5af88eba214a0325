// The blurring operator A itself as an explicit dense matrix (eq. (1.1)): the "direct"
// split Bregman of the paper's comparison (its Table 4 rows ANI A / ISO A, cost model of
// Sec. 4.3 case (i)) runs CGLS with A instead of the Kronecker-product sum.
//
// A is N x N (N = n^2), FP64, column-major: A[i + j N] is the weight of source pixel j in
// blurred pixel i.  With the PSF centre (c0, c1) = (s0/2, s1/2) and the boundary extension
// ext() of the blur kernels, blurred pixel (r, c) takes P(a, b) from source pixel
// (ext(r - a + c0), ext(c - b + c1)) for every tap; taps that fold onto the same source pixel
// (reflexive boundary) add.  Products: y = A x by column chunks (partials in a fixed order,
// then a fixed-order sum), y = A^T x by one warp per column; both FP64, deterministic.
#include "kpsb_internal.cuh"

namespace kpsb {

static constexpr int DENSE_MAX_N = 128;   // 16384^2 FP64 = 2 GiB
static constexpr int DN_T = 256;          // rows per block of the A x kernel
static constexpr int DN_CHUNK = 1024;     // columns per partial of the A x kernel

// One thread per blurred pixel i (one row of A), taps in a fixed order.
__global__ void dense_blur_kernel(const double* __restrict__ psf, int s0, int s1, int n, int bc,
                                  double* __restrict__ A) {
  const long long N = (long long)n * n;
  const int c0 = s0 / 2, c1 = s1 / 2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i % n), c = (int)(i / n);
    for (int b = 0; b < s1; ++b) {
      const int cc = ext_index(c - b + c1, n, bc);
      if (cc < 0) continue;
      for (int a = 0; a < s0; ++a) {
        const int rr = ext_index(r - a + c0, n, bc);
        if (rr < 0) continue;
        A[i + ((long long)rr + (long long)cc * n) * N] += psf[a + b * s0];
      }
    }
  }
}

size_t dense_partials(int n) {
  const long long N = (long long)n * n;
  return (size_t)((N + DN_CHUNK - 1) / DN_CHUNK) * (size_t)N;  // doubles
}

// Partials of y = A x: part[q][i] = sum_{j in chunk q} A[i + j N] x[j].  grid (row blocks,
// chunks, jobs); x of the chunk staged in shared memory.
__global__ void __launch_bounds__(DN_T) dense_ax_partial_kernel(const KPJob* __restrict__ jobs) {
  const KPJob& J = jobs[blockIdx.z];
  if (J.active && !*J.active) return;
  const long long N = (long long)J.n * J.n;
  const long long i = blockIdx.x * (long long)DN_T + threadIdx.x;
  const long long j0 = (long long)blockIdx.y * DN_CHUNK;
  if (blockIdx.x * (long long)DN_T >= N || j0 >= N) return;
  const long long j1 = j0 + DN_CHUNK < N ? j0 + DN_CHUNK : N;
  __shared__ double xs[DN_CHUNK];
  for (long long j = j0 + threadIdx.x; j < j1; j += DN_T) xs[j - j0] = J.X[j];
  __syncthreads();
  if (i >= N) return;
  const double* a = J.A + i;
  double acc = 0.0;
  for (long long j = j0; j < j1; ++j) acc = fma(a[j * N], xs[j - j0], acc);
  ((double*)J.Z)[blockIdx.y * N + i] = acc;
}

// y[i] = sum of the partials in chunk order.
__global__ void dense_ax_sum_kernel(const KPJob* __restrict__ jobs) {
  const KPJob& J = jobs[blockIdx.y];
  if (J.active && !*J.active) return;
  const long long N = (long long)J.n * J.n;
  const int nch = (int)((N + DN_CHUNK - 1) / DN_CHUNK);
  const double* part = (const double*)J.Z;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nch; ++q) s += part[q * N + i];
    J.Y[i] = s;
  }
}

// y = A^T x: warp w of the grid owns column j = w; lanes stride the rows, then a fixed
// shuffle tree.  grid (ceil(N / 8), jobs), 256 threads.
__global__ void __launch_bounds__(256) dense_atx_kernel(const KPJob* __restrict__ jobs) {
  const KPJob& J = jobs[blockIdx.y];
  if (J.active && !*J.active) return;
  const long long N = (long long)J.n * J.n;
  const long long j = blockIdx.x * 8LL + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= N) return;
  const double* a = J.A + j * N;
  double acc = 0.0;
  for (long long i = lane; i < N; i += 32) acc = fma(a[i], J.X[i], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) J.Y[j] = acc;
}

kpsb_status dense_apply_batch(const KPJob* jobs_d, int njobs, int n, int transpose, cudaStream_t st) {
  if (njobs <= 0) return KPSB_OK;
  const long long N = (long long)n * n;
  if (!transpose) {
    dim3 g1((unsigned)((N + DN_T - 1) / DN_T), (unsigned)((N + DN_CHUNK - 1) / DN_CHUNK), njobs);
    dense_ax_partial_kernel<<<g1, DN_T, 0, st>>>(jobs_d);
    KPSB_CHECK_LAUNCH();
    dim3 g2((unsigned)std::min<long long>((N + 255) / 256, 4096), njobs);
    dense_ax_sum_kernel<<<g2, 256, 0, st>>>(jobs_d);
    KPSB_CHECK_LAUNCH();
  } else {
    dim3 g((unsigned)((N + 7) / 8), njobs);
    dense_atx_kernel<<<g, 256, 0, st>>>(jobs_d);
    KPSB_CHECK_LAUNCH();
  }
  return KPSB_OK;
}

}  // namespace kpsb

using namespace kpsb;

extern "C" kpsb_status kp_dense_blur(const double* psf, int s0, int s1, int n, int bc, kpsb_kp_t* out) {
  clear_error();
  KPSB_REQUIRE(psf && out, "null pointer");
  *out = nullptr;
  KPSB_TRY(ra_check(s0, s1, n, bc));
  KPSB_REQUIRE(n <= DENSE_MAX_N, "explicit A is limited to n <= %d (got %d)", DENSE_MAX_N, n);
  const size_t N = (size_t)n * n;
  kpsb_kp* h = new kpsb_kp();
  h->n = n;
  h->k = 0;
  h->kp = 0;
  KPSB_TRY_CUDA(cudaGetDevice(&h->device));
  double* dpsf = nullptr;
  cudaError_t e = cudaMalloc((void**)&h->A_dense, sizeof(double) * N * N);
  if (e == cudaSuccess) e = cudaMalloc((void**)&dpsf, sizeof(double) * s0 * s1);
  if (e == cudaSuccess) e = cudaMemcpy(dpsf, psf, sizeof(double) * s0 * s1, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->A_dense, 0, sizeof(double) * N * N);
  if (e == cudaSuccess) {
    dense_blur_kernel<<<(unsigned)std::min<size_t>((N + 255) / 256, 4096), 256>>>(dpsf, s0, s1, n, bc, h->A_dense);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (dpsf) cudaFree(dpsf);
  if (e != cudaSuccess) {
    set_error("explicit A (%zu bytes): %s", sizeof(double) * N * N, cudaGetErrorString(e));
    kp_free(h);
    return e == cudaErrorMemoryAllocation ? KPSB_ENOMEM : KPSB_ECUDA;
  }
  *out = h;
  return KPSB_OK;
}

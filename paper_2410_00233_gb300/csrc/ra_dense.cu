// R(A) products for a general operator given as an explicit matrix (no PSF structure): the
// rearrangement of eq. (2.2) read straight from A, in single precision as the paper does
// for R(A) (Sec. 1: A replaced by its SP copy for the TSVD).
//
// A is N x N (N = n^2) column-major; its n x n block (i, j) is A_{ij}[p, q] =
// A[(i n + p) + (j n + q) N], and row i + j n of R(A) is vec(A_{ij})^T:
//   (R(A) v)[i + j n]   = sum_{p,q} A[(i n + p) + (j n + q) N] v[p + q n]
//   (R(A)^T u)[p + q n] = sum_{i,j} A[(i n + p) + (j n + q) N] u[i + j n]
// Forward: one warp per output (i, j), lanes along p (contiguous), q in order.  Transpose:
// one block per q, one thread per p (contiguous), (j, i) in order.  Both read A once per
// group of RD_VB vectors and sum in a fixed order; U = R V [+ beta * prev] as the PSF path.
#include "kpsb_internal.cuh"

namespace kpsb {

static constexpr int RD_VB = 8;  // vectors per pass over A

__global__ void __launch_bounds__(256) ra_dense_fwd_kernel(const float* __restrict__ A, int n,
                                                           const float* __restrict__ V, int ldv, int v0,
                                                           int nv, float* __restrict__ U, int ldu,
                                                           const float* __restrict__ prev, int ldp,
                                                           const double* __restrict__ beta_dev,
                                                           float beta_host, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const long long N = (long long)n * n;
  const long long o = blockIdx.x * 8LL + (threadIdx.x >> 5);  // output (i, j)
  const int lane = threadIdx.x & 31;
  if (o >= N) return;
  const int i = (int)(o % n), j = (int)(o / n);
  float acc[RD_VB];
#pragma unroll
  for (int v = 0; v < RD_VB; ++v) acc[v] = 0.f;
  for (int q = 0; q < n; ++q) {
    const float* a = A + (long long)i * n + ((long long)j * n + q) * N;
    for (int p = lane; p < n; p += 32) {
      const float av = a[p];
#pragma unroll
      for (int v = 0; v < RD_VB; ++v)
        if (v < nv) acc[v] = fmaf(av, V[(size_t)(v0 + v) * ldv + p + (size_t)q * n], acc[v]);
    }
  }
  const float beta = beta_dev ? (float)(*beta_dev) : beta_host;
#pragma unroll
  for (int v = 0; v < RD_VB; ++v) {
    float s = acc[v];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0 && v < nv) {
      if (prev) s = fmaf(beta, prev[(size_t)(v0 + v) * ldp + o], s);
      U[(size_t)(v0 + v) * ldu + o] = s;
    }
  }
}

__global__ void __launch_bounds__(256) ra_dense_adj_kernel(const float* __restrict__ A, int n,
                                                           const float* __restrict__ V, int ldv, int v0,
                                                           int nv, float* __restrict__ U, int ldu,
                                                           const float* __restrict__ prev, int ldp,
                                                           const double* __restrict__ beta_dev,
                                                           float beta_host, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const long long N = (long long)n * n;
  const int q = blockIdx.x;
  const float beta = beta_dev ? (float)(*beta_dev) : beta_host;
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    float acc[RD_VB];
#pragma unroll
    for (int v = 0; v < RD_VB; ++v) acc[v] = 0.f;
    for (int j = 0; j < n; ++j) {
      const float* a = A + p + ((long long)j * n + q) * N;
      for (int i = 0; i < n; ++i) {
        const float av = a[(long long)i * n];
#pragma unroll
        for (int v = 0; v < RD_VB; ++v)
          if (v < nv) acc[v] = fmaf(av, V[(size_t)(v0 + v) * ldv + i + (size_t)j * n], acc[v]);
      }
    }
    const long long e = p + (long long)q * n;
#pragma unroll
    for (int v = 0; v < RD_VB; ++v)
      if (v < nv) {
        float s = acc[v];
        if (prev) s = fmaf(beta, prev[(size_t)(v0 + v) * ldp + e], s);
        U[(size_t)(v0 + v) * ldu + e] = s;
      }
  }
}

kpsb_status ra_dense_apply(const float* A, int n, const float* V, int ldv, int nb, float* U, int ldu,
                           int transpose, const float* prev, int ldp, const double* beta_dev,
                           float beta_host, const int* skip, cudaStream_t st) {
  const long long N = (long long)n * n;
  for (int v0 = 0; v0 < nb; v0 += RD_VB) {
    const int nv = std::min(RD_VB, nb - v0);
    if (!transpose) {
      ra_dense_fwd_kernel<<<(unsigned)((N + 7) / 8), 256, 0, st>>>(A, n, V, ldv, v0, nv, U, ldu, prev, ldp,
                                                                  beta_dev, beta_host, skip);
    } else {
      ra_dense_adj_kernel<<<n, std::min(256, ((n + 31) / 32) * 32), 0, st>>>(A, n, V, ldv, v0, nv, U, ldu,
                                                                         prev, ldp, beta_dev, beta_host, skip);
    }
    KPSB_CHECK_LAUNCH();
  }
  return KPSB_OK;
}

}  // namespace kpsb

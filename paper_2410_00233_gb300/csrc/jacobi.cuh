// One-sided Jacobi SVD of a small FP64 matrix by one thread block (device function shared by
// the stand-alone small-SVD kernel and the one-block EGKB).
#pragma once

#include "common.cuh"

namespace kpsb {

// ---- one-sided Jacobi SVD (Hestenes) in one thread block -----------------------------------
static constexpr int JL = 8;  // lanes per column pair
// Columns p < q are rotated so that they become orthogonal; a cyclic "round robin"
// ordering visits every pair once per sweep, the disjoint pairs of a round at the same time
// (JL lanes each).
// After convergence the column norms are the singular values, the normalised columns the
// left singular vectors and the accumulated rotations the right singular vectors.
// Called by every thread of a block (any multiple of 32 threads); smem holds
// m * nc + nc * nc doubles.  Ends with the block synchronised.
__device__ __forceinline__ void jacobi_svd_block(const double* __restrict__ A, int lda, int m, int nc,
                                                 double* __restrict__ U, double* __restrict__ S,
                                                 double* __restrict__ V, int* __restrict__ sweeps_out,
                                                 int max_sweeps, double* smem) {
  double* a = smem;            // m x nc, ld m
  double* v = a + m * nc;      // nc x nc, ld nc
  __shared__ int rot_count;
  __shared__ double nrm[64];
  __shared__ int perm[64];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  for (int e = tid; e < m * nc; e += blockDim.x) a[e] = A[(e % m) + (size_t)(e / m) * lda];
  for (int e = tid; e < nc * nc; e += blockDim.x) v[e] = (e % nc == e / nc) ? 1.0 : 0.0;
  __syncthreads();
  const int ncp = nc + (nc & 1);
  const double tol = fmax((double)m, 8.0) * 2.220446049250313e-16;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) rot_count = 0;
    __syncthreads();
    for (int round = 0; round < ncp - 1; ++round) {
      // JL lanes per column pair, 32 / JL pairs per warp: GB300 issues FP64 instructions to a
      // narrow pipe, so every warp instruction should carry as many useful lanes as possible
      for (int pb = warp * (32 / JL); pb < ncp / 2; pb += nwarps * (32 / JL)) {
        const int pi = pb + lane / JL, sl = lane % JL;
        int p = 0, q = 0;
        bool act = pi < ncp / 2;
        if (act) {
          const int pos_a = pi, pos_b = ncp - 1 - pi;
          p = pos_a == 0 ? 0 : 1 + (pos_a - 1 + round) % (ncp - 1);
          q = 1 + (pos_b - 1 + round) % (ncp - 1);
          act = p < nc && q < nc;
          if (p > q) { int t = p; p = q; q = t; }
        }
        double al = 0.0, be = 0.0, ga = 0.0;
        if (act) {
          for (int r = sl; r < m; r += JL) {
            double x = a[r + p * m], y = a[r + q * m];
            al = fma(x, x, al);
            be = fma(y, y, be);
            ga = fma(x, y, ga);
          }
        }
#pragma unroll
        for (int o = JL / 2; o > 0; o >>= 1) {  // butterfly inside the JL-lane group
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (act && fabs(ga) > tol * sqrt(al * be) && ga != 0.0) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          for (int r = sl; r < m; r += JL) {
            double x = a[r + p * m], y = a[r + q * m];
            a[r + p * m] = c * x - s * y;
            a[r + q * m] = s * x + c * y;
          }
          for (int r = sl; r < nc; r += JL) {
            double x = v[r + p * nc], y = v[r + q * nc];
            v[r + p * nc] = c * x - s * y;
            v[r + q * nc] = s * x + c * y;
          }
          if (sl == 0) atomicAdd(&rot_count, 1);
        }
      }
      __syncthreads();
    }
    if (rot_count == 0) break;
    __syncthreads();
  }
  for (int j = warp; j < nc; j += nwarps) {
    double s2 = 0.0;
    for (int r = lane; r < m; r += 32) s2 = fma(a[r + j * m], a[r + j * m], s2);
    s2 = warp_sum(s2);
    if (lane == 0) nrm[j] = sqrt(s2);
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < nc; ++j) perm[j] = j;
    for (int i = 0; i < nc; ++i) {  // selection sort, descending, stable on ties
      int best = i;
      for (int j = i + 1; j < nc; ++j)
        if (nrm[perm[j]] > nrm[perm[best]]) best = j;
      int t = perm[i]; perm[i] = perm[best]; perm[best] = t;
    }
    if (sweeps_out) *sweeps_out = sweep + 1;
  }
  __syncthreads();
  for (int e = tid; e < m * nc; e += blockDim.x) {
    int r = e % m, j = e / m, src = perm[j];
    double sj = nrm[src];
    U[e] = sj > 0.0 ? a[r + src * m] / sj : 0.0;
  }
  for (int e = tid; e < nc * nc; e += blockDim.x) V[e] = v[(e % nc) + perm[e / nc] * nc];
  for (int j = tid; j < nc; j += blockDim.x) S[j] = nrm[perm[j]];
  __syncthreads();
}

}  // namespace kpsb

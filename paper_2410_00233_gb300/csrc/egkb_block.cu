// One-block EGKB (Alg. 1) for small images: the whole Golub-Kahan recurrence of one problem
// with its reorthogonalisation (steps 3-13), the FP64 SVD of the lower bidiagonal C (step 15),
// the Ritz vectors (steps 16-17) and the terms with their sign convention (Theorem 2.1)
// run in one thread block, every problem of a batch in the same two launches.  R(A) is
// applied through the PSF's index map (Sec. 2.1, eq. (2.2)): U = R(A) V is
//   reduce : D_a = sum of V over the (anti-)diagonals that feed tap a,
//   mix    : w_b = sum_a P(a, b) D_a,
//   expand : U[i + j n] = sum of w_b over the taps b with j = ext(i - b + c1),
// and R(A)^T swaps the roles of the two PSF directions.
// Arithmetic classes follow the multi-kernel path: FP32 vectors and products, FP32 partial
// sums per thread and warp, FP64 sums across warps, FP64 recurrence scalars, mixing and SVD.
// Every reduction has a fixed order, so a problem gives the same bits alone and in a batch.
#include <math.h>
#include <string.h>

#include "jacobi.cuh"
#include "kpsb_internal.cuh"

namespace kpsb {

static constexpr int EB_T = 512;           // threads per block (two blocks per SM)
static constexpr int EB_W = EB_T / 32;
static constexpr int EB_DB = 8;            // basis columns per dot-product chunk
static constexpr int EB_MAX_N = 128;
static constexpr int EB_MAX_S = 128;       // PSF side
static constexpr int EB_MAX_PSF = 4096;    // PSF entries staged in shared memory
static constexpr int EB_KP = 64;           // largest k_p of the build
static constexpr int EB_LD = EB_KP + 2;    // leading dimension of the small matrices
static constexpr int EB_SMALL = 3 * EB_LD * EB_KP + EB_LD;  // C, U, V (and sigma), doubles

bool eb_eligible(int n, int s0, int s1) {
  return n >= 2 && n <= EB_MAX_N && s0 <= EB_MAX_S && s1 <= EB_MAX_S && s0 * s1 <= EB_MAX_PSF;
}

struct EbInfo {  // per problem, read by the host between the two launches
  int nq, ns, ksel, finished, kk, pad[3];
  double bytes;  // algorithmic bytes of the R(A) products and CGS2 passes (as the TSVD timers)
  double sigma[EB_KP];
};

struct EbJob {
  const float* psf;
  int s0, s1, n, bc;
  EgkbParams P;
  int full_reorth, kpmax;
  float* S;       // n^2 x (kpmax + 1): s_1, s_2, ...
  float* Q;       // n^2 x (kpmax + 1): q_1, q_2, ...
  double* small;  // C (m x nc), U (m x nc), V (nc x nc) at strides EB_LD * EB_KP, then sigma
  EbInfo* info;
  float* Ax;      // handle arrays for the terms (null: the problem failed)
  float* Ay;
  double* sigma_out;
};

// Recurrence scalars (the device-side state of the multi-kernel path, in shared memory).
struct EbState {
  double alpha[EB_KP + 4], t[EB_KP + 4], zeta[EB_KP + 4], nu[EB_KP + 4];
  double norm, coef_s, coef_q, bnorm;
  double bytes;  // algorithmic bytes so far: R(A) products and CGS2 passes
  int nq, ns, k_sel, kp_target, finished, stop;
};

// Algorithmic bytes of one R(A) product of one vector (read V, write U, read prev when given,
// the PSF) and of one CGS2 against m basis vectors (two passes: the basis read twice and v
// three times per pass; a plain norm when m = 0), the same counts as the multi-kernel path's
// TSVD timers.
__device__ __forceinline__ double eb_ra_bytes(int N, bool prev, int s0, int s1) {
  return 4.0 * N * (prev ? 3.0 : 2.0) + 4.0 * s0 * s1;
}
__device__ __forceinline__ double eb_cgs2_bytes(int N, int m) {
  return m > 0 ? 2.0 * (2.0 * m + 3.0) * N * 4.0 : 4.0 * N;
}

// ---- block-level building blocks (every thread calls; each ends synchronised) ---------------

// ||v||_2: FP32 squares in two interleaved accumulators per thread, FP64 across threads.
__device__ __forceinline__ double eb_norm(const float* __restrict__ v, int N, double* red) {
  float s0 = 0.f, s1 = 0.f;
  int e = threadIdx.x;
  for (; e + EB_T < N; e += 2 * EB_T) {
    const float a = v[e], b = v[e + EB_T];
    s0 = fmaf(a, a, s0);
    s1 = fmaf(b, b, s1);
  }
  if (e < N) s0 = fmaf(v[e], v[e], s0);
  return sqrt(block_sum<double>((double)(s0 + s1), red));
}

// v *= 1 / nrm (zero norm clears v).
__device__ __forceinline__ void eb_scale(float* __restrict__ v, int N, double nrm) {
  const float s = nrm > 0.0 ? (float)(1.0 / nrm) : 0.f;
  for (int e = threadIdx.x; e < N; e += EB_T) v[e] *= s;
  __syncthreads();
}

// Sum of V over one diagonal (r - q = d) or anti-diagonal (r + q = sg) by one warp.
__device__ __forceinline__ float eb_diag(const float* __restrict__ V, int n, int d, int lane) {
  float acc = 0.f;
  const int r_lo = d > 0 ? d : 0, r_hi = d < 0 ? n + d : n;
  for (int r = r_lo + lane; r < r_hi; r += 32) acc += V[r + (r - d) * n];
  return warp_sum(acc);
}
__device__ __forceinline__ float eb_anti(const float* __restrict__ V, int n, int sg, int lane) {
  float acc = 0.f;
  const int r_lo = sg - (n - 1) > 0 ? sg - (n - 1) : 0, r_hi = sg < n - 1 ? sg : n - 1;
  for (int r = r_lo + lane; r <= r_hi; r += 32) acc += V[r + (sg - r) * n];
  return warp_sum(acc);
}

// U = R(A) V (transpose: R(A)^T V) [+ beta prev].
__device__ void eb_ra(const float* __restrict__ psf, int s0, int s1, int n, int bc, const float* V,
                      float* U, const float* prev, float beta, bool transpose, double* Dsh, float* wsh) {
  const int s_red = transpose ? s1 : s0, c_red = s_red / 2;
  const int s_exp = transpose ? s0 : s1, c_exp = s_exp / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // reduce: tap t collects the diagonal r - q = t - c_red and, reflexive, the anti-diagonals
  // r + q = t - 1 - c_red and t - 1 - c_red + 2n (mirrored indices)
  for (int t = warp; t < s_red; t += EB_W) {
    double D = (double)eb_diag(V, n, t - c_red, lane);
    if (bc == KPSB_BC_REFLEXIVE) {
      const int sg = t - 1 - c_red;
      if (sg >= 0 && sg <= 2 * n - 2) D += (double)eb_anti(V, n, sg, lane);
      if (sg + 2 * n <= 2 * n - 2) D += (double)eb_anti(V, n, sg + 2 * n, lane);
    }
    if (lane == 0) Dsh[t] = D;
  }
  __syncthreads();
  // mix (FP64): R: w_b = sum_a P(a, b) D_a;  R^T: w_a = sum_b P(a, b) D_b  (P column-major s0 x s1)
  for (int o = threadIdx.x; o < s_exp; o += EB_T) {
    double acc = 0.0;
    if (!transpose) {
      for (int a = 0; a < s_red; ++a) acc += (double)psf[a + o * s0] * Dsh[a];
    } else {
      for (int b = 0; b < s_red; ++b) acc += (double)psf[o + b * s0] * Dsh[b];
    }
    wsh[o] = (float)acc;
  }
  __syncthreads();
  // expand: U[i + j n] = sum over taps t with j = ext(i - t + c_exp) of w_t
  const int N = n * n;
  int i = threadIdx.x % n, j = threadIdx.x / n;
  const int di = EB_T % n, dj = EB_T / n;
  for (int e = threadIdx.x; e < N; e += EB_T) {
    float acc = 0.f;
    int t = i - j + c_exp;
    if (t >= 0 && t < s_exp) acc += wsh[t];
    if (bc == KPSB_BC_REFLEXIVE) {
      t = i + j + 1 + c_exp;
      if (t < s_exp) acc += wsh[t];
      t -= 2 * n;
      if (t >= 0 && t < s_exp) acc += wsh[t];
    }
    if (prev) acc = fmaf(beta, prev[e], acc);
    U[e] = acc;
    i += di;
    j += dj;
    if (i >= n) {
      i -= n;
      ++j;
    }
  }
  __syncthreads();
}

// CGS2: two passes of v -= B (B^T v) against the m columns of B (ld N); returns ||v|| after
// the second pass (after none when m = 0).
__device__ double eb_cgs2(const float* __restrict__ B, int m, float* v, int N, float (*wpart)[EB_DB],
                          double* hd, float* hf, double* red) {
  if (m <= 0) return eb_norm(v, N, red);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float ss0 = 0.f, ss1 = 0.f;
  for (int pass = 0; pass < 2; ++pass) {
    // h = B^T v by chunks of EB_DB columns: two interleaved FP32 accumulators per thread and
    // column, a warp butterfly, the warp totals in FP64 in a fixed order
    for (int c0 = 0; c0 < m; c0 += EB_DB) {
      float a0[EB_DB], a1[EB_DB];
#pragma unroll
      for (int u = 0; u < EB_DB; ++u) a0[u] = a1[u] = 0.f;
      int e = threadIdx.x;
      for (; e + EB_T < N; e += 2 * EB_T) {
        const float x = v[e], y = v[e + EB_T];
#pragma unroll
        for (int u = 0; u < EB_DB; ++u)
          if (c0 + u < m) {
            const float* b = B + (size_t)(c0 + u) * N;
            a0[u] = fmaf(b[e], x, a0[u]);
            a1[u] = fmaf(b[e + EB_T], y, a1[u]);
          }
      }
      if (e < N) {
        const float x = v[e];
#pragma unroll
        for (int u = 0; u < EB_DB; ++u)
          if (c0 + u < m) a0[u] = fmaf(B[e + (size_t)(c0 + u) * N], x, a0[u]);
      }
#pragma unroll
      for (int u = 0; u < EB_DB; ++u) {
        const float t = warp_sum(a0[u] + a1[u]);
        if (lane == 0) wpart[warp][u] = t;
      }
      __syncthreads();
      if (threadIdx.x < EB_DB && c0 + (int)threadIdx.x < m) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < EB_W; ++w) t += (double)wpart[w][threadIdx.x];
        hd[c0 + threadIdx.x] = t;
        hf[c0 + threadIdx.x] = (float)t;
      }
      __syncthreads();
    }
    // v -= B h (FP32, columns in order), two elements per iteration so that twice as many
    // basis loads are in flight
    ss0 = ss1 = 0.f;
    int e = threadIdx.x;
    for (; e + EB_T < N; e += 2 * EB_T) {
      float c0r = 0.f, c1r = 0.f;
#pragma unroll 4
      for (int c = 0; c < m; ++c) {
        const float* b = B + (size_t)c * N;
        c0r = fmaf(b[e], hf[c], c0r);
        c1r = fmaf(b[e + EB_T], hf[c], c1r);
      }
      const float x0 = v[e] - c0r, x1 = v[e + EB_T] - c1r;
      v[e] = x0;
      v[e + EB_T] = x1;
      ss0 = fmaf(x0, x0, ss0);
      ss1 = fmaf(x1, x1, ss1);
    }
    if (e < N) {
      float corr = 0.f;
      for (int c = 0; c < m; ++c) corr = fmaf(B[e + (size_t)c * N], hf[c], corr);
      const float x = v[e] - corr;
      v[e] = x;
      ss0 = fmaf(x, x, ss0);
    }
    __syncthreads();
  }
  return sqrt(block_sum<double>((double)(ss0 + ss1), red));
}

// Decision after t_j (the s-phase of step j; j = 1 is the start vector).
__device__ __forceinline__ void eb_after_t(EbState& s, const EgkbParams& P, int j, double tj) {
  int stop = 0;
  if (j == 1) {
    s.t[1] = tj;
    s.ns = 1;
    if (!(tj > 0.0)) {
      s.finished = 2;
      tj = 0.0;
      stop = 1;
    }
  } else {
    s.bnorm = fmax(s.bnorm, tj);
    if (!(tj > P.bd_tol * s.bnorm)) {  // invariant subspace: s_j = 0, C's last row 0
      s.t[j] = 0.0;
      tj = 0.0;
      s.ns = j;
      s.finished = 2;
      stop = 1;
    } else {
      s.t[j] = tj;
      s.ns = j;
      if (s.kp_target > 0 && s.nq >= s.kp_target) {
        s.finished = 1;
        stop = 1;
      }
    }
  }
  s.norm = tj;
  s.coef_q = -s.t[j];
  s.stop = stop;
}

// Decision after alpha_j (the q-phase of step j): the nu rule of Sec. 2.2 (eq. (2.6)).
__device__ __forceinline__ void eb_after_alpha(EbState& s, const EgkbParams& P, int j, double aj) {
  s.norm = aj;
  s.bnorm = fmax(s.bnorm, aj);
  if (!(aj > P.bd_tol * s.bnorm) || (j == 1 && !(aj > 0.0))) {
    s.finished = 3;  // q_j is not accepted
    s.stop = 1;
    return;
  }
  s.alpha[j] = aj;
  s.nq = j;
  s.coef_s = -aj;
  if (j >= 2) {
    s.zeta[j] = aj * s.t[j];
    if (j >= 3) s.nu[j] = sqrt(s.zeta[j] * s.zeta[j - 1]);
  }
  if (P.k_fixed <= 0 && s.k_sel < 0 && j >= 4) {
    const int i = j - 1;
    const int kmin = P.k_min > 3 ? P.k_min : 3;
    if (i >= kmin && (s.nu[j] > s.nu[i] || s.nu[i] < P.tau * s.nu[3]))
      s.k_sel = i;
    else if (i >= P.k_cap)
      s.k_sel = P.k_cap;
    if (s.k_sel >= 0) {
      const int kp = s.k_sel + P.p;
      s.kp_target = kp > s.nq ? kp : s.nq;
    }
  }
  s.stop = 0;
}

// ---- launch 1: the recurrence and the SVD of C, one block per problem ------------------------
__global__ void __launch_bounds__(EB_T, 2) egkb_block_kernel(const EbJob* __restrict__ jobs) {
  extern __shared__ double dsm[];  // Jacobi scratch: m nc + nc nc doubles
  __shared__ float psf[EB_MAX_PSF];
  __shared__ double Dsh[EB_MAX_S];
  __shared__ float wsh[EB_MAX_S];
  __shared__ float wpart[EB_W][EB_DB];
  __shared__ double hd[EB_KP + 2];
  __shared__ float hf[EB_KP + 2];
  __shared__ double red[32];
  __shared__ EbState es;
  const EbJob J = jobs[blockIdx.x];
  const int n = J.n, N = n * n, tid = threadIdx.x;
  for (int e = tid; e < J.s0 * J.s1; e += EB_T) psf[e] = J.psf[e];
  if (tid == 0) {
    memset(&es, 0, sizeof(EbState));
    es.k_sel = J.P.k_fixed > 0 ? J.P.k_fixed : -1;
    es.kp_target = J.P.k_fixed > 0 ? J.P.k_fixed + J.P.p : -1;
  }
  __syncthreads();
  float* S = J.S;
  float* Q = J.Q;
  // s_1 = y / ||y||  (y written into S[:, 0] before the launch)
  double nrm = eb_norm(S, N, red);
  if (tid == 0) eb_after_t(es, J.P, 1, nrm);
  __syncthreads();
  eb_scale(S, N, es.norm);
  bool stop = es.stop;
  if (!stop) {  // q_1 = R^T s_1 / alpha_1
    eb_ra(psf, J.s0, J.s1, n, J.bc, S, Q, nullptr, 0.f, true, Dsh, wsh);
    nrm = eb_norm(Q, N, red);
    if (tid == 0) {
      es.bytes += eb_ra_bytes(N, false, J.s0, J.s1);
      eb_after_alpha(es, J.P, 1, nrm);
    }
    __syncthreads();
    eb_scale(Q, N, es.norm);
    stop = es.stop;
  }
  for (int j = 2; j <= J.kpmax + 1 && !stop; ++j) {
    float* sj = S + (size_t)(j - 1) * N;
    float* sjm1 = S + (size_t)(j - 2) * N;
    float* qjm1 = Q + (size_t)(j - 2) * N;
    float* qj = Q + (size_t)(j - 1) * N;
    // s-phase: s_j = R q_{j-1} - alpha_{j-1} s_{j-1}, reorthogonalised, t_j
    eb_ra(psf, J.s0, J.s1, n, J.bc, qjm1, sj, sjm1, (float)es.coef_s, false, Dsh, wsh);
    nrm = eb_cgs2(S, J.full_reorth ? j - 1 : 0, sj, N, wpart, hd, hf, red);
    if (tid == 0) {
      es.bytes += eb_ra_bytes(N, true, J.s0, J.s1) + eb_cgs2_bytes(N, J.full_reorth ? j - 1 : 0);
      eb_after_t(es, J.P, j, nrm);
    }
    __syncthreads();
    eb_scale(sj, N, es.norm);
    stop = es.stop;
    if (stop || j == J.kpmax + 1) break;  // only s_{kp+1} is needed from the last step
    // q-phase: q_j = R^T s_j - t_j q_{j-1}, reorthogonalised, alpha_j and the nu rule
    eb_ra(psf, J.s0, J.s1, n, J.bc, sj, qj, qjm1, (float)es.coef_q, true, Dsh, wsh);
    nrm = eb_cgs2(Q, j - 1, qj, N, wpart, hd, hf, red);
    if (tid == 0) {
      es.bytes += eb_ra_bytes(N, true, J.s0, J.s1) + eb_cgs2_bytes(N, j - 1);
      eb_after_alpha(es, J.P, j, nrm);
    }
    __syncthreads();
    eb_scale(qj, N, es.norm);
    stop = es.stop;
  }
  const int nq = es.nq;
  const int kk = es.k_sel > 0 ? min(es.k_sel, nq) : min(J.P.k_cap, nq);
  if (tid == 0) {
    J.info->nq = nq;
    J.info->ns = es.ns;
    J.info->ksel = es.k_sel;
    J.info->finished = es.finished;
    J.info->kk = nq >= 1 ? kk : 0;
    J.info->bytes = es.bytes;
  }
  if (nq < 1) return;
  // C ((nq + 1) x nq lower bidiagonal) and its FP64 SVD (step 15)
  const int m = nq + 1, nc = nq;
  double* C = J.small;
  double* U = C + EB_LD * EB_KP;
  double* V = U + EB_LD * EB_KP;
  double* sg = V + EB_LD * EB_KP;
  for (int e = tid; e < m * nc; e += EB_T) {
    const int r = e % m, c = e / m;
    C[e] = r == c ? es.alpha[c + 1] : r == c + 1 ? es.t[c + 2] : 0.0;
  }
  __syncthreads();
  jacobi_svd_block(C, m, m, nc, U, sg, V, nullptr, 60, dsm);
  for (int e = tid; e < kk; e += EB_T) J.info->sigma[e] = sg[e];
}

// ---- launch 2: Ritz vectors and terms, one block per problem ---------------------------------
// Ax = S_{nq+1} U_C[:, :k], Ay = Q_nq V_C[:, :k] (FP32 products in column order, as the
// multi-kernel path), then the sign convention: the first entry of largest magnitude of
// vec(Ay_i) is made positive, Ax_i flipped with it.
__global__ void __launch_bounds__(EB_T) egkb_terms_kernel(const EbJob* __restrict__ jobs) {
  __shared__ float Tu[EB_LD * EB_KP];
  __shared__ float Tv[EB_LD * EB_KP];
  __shared__ unsigned long long wkey[EB_W];
  __shared__ int flip[EB_KP];
  const EbJob J = jobs[blockIdx.x];
  if (!J.Ax) return;
  const int n = J.n, N = n * n, tid = threadIdx.x;
  const int nq = J.info->nq, kk = J.info->kk, m = nq + 1, nc = nq;
  const double* U = J.small + EB_LD * EB_KP;
  const double* V = U + EB_LD * EB_KP;
  for (int e = tid; e < m * kk; e += EB_T) Tu[(e % m) + (e / m) * EB_LD] = (float)U[(e % m) + (size_t)(e / m) * m];
  for (int e = tid; e < nc * kk; e += EB_T) Tv[(e % nc) + (e / nc) * EB_LD] = (float)V[(e % nc) + (size_t)(e / nc) * nc];
  __syncthreads();
  for (int side = 0; side < 2; ++side) {
    const float* Y = side == 0 ? J.S : J.Q;
    const float* T = side == 0 ? Tu : Tv;
    const int mm = side == 0 ? m : nc;
    float* Out = side == 0 ? J.Ax : J.Ay;
    for (int r = tid; r < N; r += EB_T) {
      for (int j0 = 0; j0 < kk; j0 += 16) {
        float acc[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] = 0.f;
        for (int i = 0; i < mm; ++i) {
          const float y = Y[r + (size_t)i * N];
#pragma unroll
          for (int u = 0; u < 16; ++u) acc[u] = fmaf(y, T[i + (j0 + u) * EB_LD], acc[u]);
        }
#pragma unroll
        for (int u = 0; u < 16; ++u)
          if (j0 + u < kk) Out[r + (size_t)(j0 + u) * N] = acc[u];
      }
    }
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  for (int j = 0; j < kk; ++j) {
    const float* ay = J.Ay + (size_t)j * N;
    unsigned long long best = 0;
    for (int e = tid; e < N; e += EB_T) {
      const unsigned long long key =
          ((unsigned long long)__float_as_uint(fabsf(ay[e])) << 32) | (0xFFFFFFFFull - (unsigned long long)e);
      best = key > best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
      best = other > best ? other : best;
    }
    if (lane == 0) wkey[warp] = best;
    __syncthreads();
    if (tid == 0) {
      unsigned long long b = 0;
      for (int w = 0; w < EB_W; ++w) b = wkey[w] > b ? wkey[w] : b;
      const long long idx = (long long)(0xFFFFFFFFull - (b & 0xFFFFFFFFull));
      flip[j] = ay[idx] < 0.f;
    }
    __syncthreads();
  }
  for (int j = 0; j < kk; ++j) {
    if (!flip[j]) continue;
    float* ax = J.Ax + (size_t)j * N;
    float* ay = J.Ay + (size_t)j * N;
    for (int e = tid; e < N; e += EB_T) {
      ax[e] = -ax[e];
      ay[e] = -ay[e];
    }
  }
  for (int j = tid; j < kk; j += EB_T) J.sigma_out[j] = J.info->sigma[j];
}

static size_t eb_a256(size_t x) { return (x + 255) / 256 * 256; }

kpsb_status egkb_block_build(const EbProblem* pr, int count, kpsb_kp_t* outs, kpsb_status* st_out,
                             std::string* msg_out, cudaStream_t st) {
  if (count <= 0) return KPSB_OK;
  for (int p = 0; p < count; ++p) {
    outs[p] = nullptr;
    st_out[p] = KPSB_OK;
    KPSB_REQUIRE(eb_eligible(pr[p].n, pr[p].s0, pr[p].s1) && pr[p].kpmax >= 1 && pr[p].kpmax <= EB_KP,
                 "one-block EGKB: problem %d outside its limits", p);
  }
  // device layout: jobs, infos, PSFs (one upload), then per problem the bases and the small
  // matrices
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off += eb_a256(b);
    return o;
  };
  const size_t o_jobs = take(sizeof(EbJob) * count);
  const size_t o_info = take(sizeof(EbInfo) * count);
  std::vector<size_t> o_psf(count), o_S(count), o_small(count);
  const size_t psf_lo = off;
  for (int p = 0; p < count; ++p) o_psf[p] = take(sizeof(float) * pr[p].s0 * pr[p].s1);
  const size_t psf_hi = off;
  for (int p = 0; p < count; ++p) {
    const size_t N = (size_t)pr[p].n * pr[p].n;
    o_S[p] = take(sizeof(float) * N * (pr[p].kpmax + 1) * 2);
    o_small[p] = take(sizeof(double) * EB_SMALL);
  }
  char* base = nullptr;
  KPSB_TRY_CUDA(cudaMallocAsync((void**)&base, off, st));
  kpsb_status s = KPSB_OK;
  std::vector<EbJob> jobs(count);
  std::vector<EbInfo> info(count);
  int dyn = 0;
  do {
    std::vector<float> pst((psf_hi - psf_lo) / sizeof(float), 0.f);
    for (int p = 0; p < count; ++p) {
      float* d = pst.data() + (o_psf[p] - psf_lo) / sizeof(float);
      for (int e = 0; e < pr[p].s0 * pr[p].s1; ++e) d[e] = (float)pr[p].psf[e];
      const size_t N = (size_t)pr[p].n * pr[p].n;
      EbJob& J = jobs[p];
      J.psf = (const float*)(base + o_psf[p]);
      J.s0 = pr[p].s0;
      J.s1 = pr[p].s1;
      J.n = pr[p].n;
      J.bc = pr[p].bc;
      J.P = pr[p].P;
      J.full_reorth = pr[p].full_reorth;
      J.kpmax = pr[p].kpmax;
      J.S = (float*)(base + o_S[p]);
      J.Q = J.S + N * (pr[p].kpmax + 1);
      J.small = (double*)(base + o_small[p]);
      J.info = (EbInfo*)(base + o_info) + p;
      J.Ax = J.Ay = nullptr;
      J.sigma_out = nullptr;
      const int kp = pr[p].kpmax;
      dyn = std::max(dyn, (int)(sizeof(double) * ((kp + 1) * kp + kp * kp)));
    }
    cudaError_t e = cudaSuccess;
    if (psf_hi > psf_lo) e = cudaMemcpyAsync(base + psf_lo, pst.data(), psf_hi - psf_lo, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_jobs, jobs.data(), sizeof(EbJob) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_info, 0, sizeof(EbInfo) * count, st);
    for (int p = 0; p < count && e == cudaSuccess; ++p) {  // start vectors into S[:, 0]
      const long long N = (long long)pr[p].n * pr[p].n;
      if (pr[p].start_host) {
        e = cudaMemcpyAsync(jobs[p].S, pr[p].start_host, sizeof(float) * N, cudaMemcpyHostToDevice, st);
      } else if ((s = la_randn<float>(jobs[p].S, N, pr[p].seed, st)) != KPSB_OK) {
        break;
      }
    }
    if (s) break;
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(egkb_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, std::max(dyn, 1));
    if (e != cudaSuccess) {
      set_error("one-block EGKB setup: %s", cudaGetErrorString(e));
      s = KPSB_ECUDA;
      break;
    }
    const int slot = timer_begin(st);
    egkb_block_kernel<<<count, EB_T, std::max(dyn, 1), st>>>((const EbJob*)(base + o_jobs));
    count_launch();
    e = cudaGetLastError();
    timer_end(slot, st, TIMER_EGKB_BLOCK, 0.0, 1);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(info.data(), base + o_info, sizeof(EbInfo) * count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error("one-block EGKB: %s", cudaGetErrorString(e));
      s = KPSB_ECUDA;
      break;
    }
    double bytes = 0.0;
    for (int p = 0; p < count; ++p) bytes += info[p].bytes;
    timer_set_value(slot, bytes);
    // handles sized by the selected rank
    for (int p = 0; p < count; ++p) {
      if (info[p].nq < 1) {
        st_out[p] = KPSB_EBREAKDOWN;
        if (msg_out) msg_out[p] = "EGKB: R(A) applied to the start vector vanishes";
        continue;
      }
      kpsb_kp* h = nullptr;
      const kpsb_status hs = kp_handle_alloc(&h, pr[p].n, info[p].kk, info[p].nq);
      if (hs != KPSB_OK) {
        st_out[p] = hs;
        if (msg_out) msg_out[p] = kpsb_last_error();
        continue;
      }
      h->sigma.assign(info[p].sigma, info[p].sigma + info[p].kk);
      jobs[p].Ax = h->Ax;
      jobs[p].Ay = h->Ay;
      jobs[p].sigma_out = h->sigma_d;
      outs[p] = h;
    }
    e = cudaMemcpyAsync(base + o_jobs, jobs.data(), sizeof(EbJob) * count, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      set_error("one-block EGKB: %s", cudaGetErrorString(e));
      s = KPSB_ECUDA;
      break;
    }
    egkb_terms_kernel<<<count, EB_T, 0, st>>>((const EbJob*)(base + o_jobs));
    count_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error("one-block EGKB terms: %s", cudaGetErrorString(e));
      s = KPSB_ECUDA;
      break;
    }
  } while (0);
  cudaFreeAsync(base, st);
  if (s != KPSB_OK) {  // a launch-level failure: no problem keeps a handle
    for (int p = 0; p < count; ++p) {
      if (outs[p]) kp_free(outs[p]);
      outs[p] = nullptr;
      st_out[p] = s;
    }
    return s;
  }
  for (int p = 0; p < count; ++p)
    if (st_out[p] != KPSB_OK) {
      if (msg_out) set_error("%s", msg_out[p].c_str());
      return st_out[p];
    }
  return KPSB_OK;
}

}  // namespace kpsb

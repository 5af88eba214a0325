// Matrix-free R(A) (Sec. 2.1, eq. (2.2)) through the PSF's index map, its dense
// materialisation, and the exact blur A (Sec. 1).
//
// Structure used (derived from the definition of the blur): with M_t the n x n matrix of
// one PSF tap, (M_t)[r, ext(r - t + c)] = 1, the blur is A = sum_{a,b} P(a,b) M_b (x) M_a,
// so R(A) = Kx P^T Ky^T with Kx[:, b] = vec(M_b), Ky[:, a] = vec(M_a).  One block apply
// U = R(A) V therefore is
//   reduce : D_a = sum_{(r,q): q = ext(r - a + c0)} V[r + q n]      (Ky^T V)
//   mix    : w_b = sum_a P(a, b) D_a                                 (P^T D)
//   expand : U[i + j n] = sum_{b: j = ext(i - b + c1)} w_b           (Kx w)
// and R(A)^T swaps the roles of (a, s0) and (b, s1) and uses P instead of P^T.
// An element (r, q) feeds tap t = r - q + c (its diagonal), and for the reflexive
// boundary also t = r + q + 1 + c and t = r + q + 1 + c - 2n (its anti-diagonal), when
// those lie in [0, s).
#include "kpsb_internal.cuh"

namespace kpsb {

static constexpr int RA_TS = 64;            // tile side of the reduction
static constexpr int RA_SLOTS = 256;        // 127 diagonal + 127 anti-diagonal slots (+2 pad)
static constexpr int RA_MAX_S = 1024;       // largest PSF side handled
static constexpr int RA_MIX_SMEM = 4096;    // PSF entries staged in shared memory for the mix (64 x 64)

__device__ __forceinline__ bool ra_tile_direct(int tr, int tq, int c, int s) {
  int dlo = (tr - tq) * RA_TS - (RA_TS - 1) + c, dhi = (tr - tq) * RA_TS + (RA_TS - 1) + c;
  return dhi >= 0 && dlo < s;
}
__device__ __forceinline__ bool ra_tile_anti(int tr, int tq, int c, int s, int n) {
  int slo = (tr + tq) * RA_TS, shi = slo + 2 * RA_TS - 2;
  // low mirror: t = S + 1 + c < s  <=>  S <= s - 2 - c
  bool lo = slo <= s - 2 - c;
  // high mirror: t = S + 1 + c - 2n in [0, s)  <=>  S in [2n - 1 - c, 2n - 2 - c + s]
  bool hi = shi >= 2 * n - 1 - c && slo <= 2 * n - 2 - c + s;
  return lo || hi;
}

// One 64x64 tile of one column of V: diagonal and anti-diagonal partial sums.  The last
// block of each column combines the partials (fixed order) into D, mixes with P and
// writes w.
template <typename T>
__global__ void __launch_bounds__(256) ra_reduce_kernel(
    const T* __restrict__ V, int ldv, int n, int bc, int s_red, int c_red, int s_exp,
    const T* __restrict__ psf, int s0, int transpose, T* __restrict__ part,
    unsigned int* __restrict__ counters, T* __restrict__ wout) {
  __shared__ T tile[RA_TS * (RA_TS + 1)];
  __shared__ double Dsh[RA_MAX_S];
  // the PSF, staged for the mix when it fits (single precision only: the FP64 tile and
  // sums already take most of the static shared memory)
  constexpr int MIX_N = sizeof(T) == sizeof(float) ? RA_MIX_SMEM : 1;
  __shared__ T Psh[MIX_N];
  const int nt = (n + RA_TS - 1) / RA_TS;
  const int ntiles = nt * nt;
  const int tr = blockIdx.x % nt, tq = blockIdx.x / nt;
  const int col = blockIdx.y;
  const T* v = V + (size_t)col * ldv;
  T* mypart = part + ((size_t)col * ntiles + blockIdx.x) * RA_SLOTS;
  const bool rel_d = ra_tile_direct(tr, tq, c_red, s_red);
  const bool rel_a = bc == KPSB_BC_REFLEXIVE && ra_tile_anti(tr, tq, c_red, s_red, n);
  if (rel_d || rel_a) {
    const int rl = threadIdx.x & 63, q0 = threadIdx.x >> 6;
    const int r = tr * RA_TS + rl;
    for (int ql = q0; ql < RA_TS; ql += 4) {
      int q = tq * RA_TS + ql;
      tile[ql * (RA_TS + 1) + rl] = (r < n && q < n) ? v[r + (size_t)q * n] : (T)0;
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (t < 2 * RA_TS - 1) {
      if (rel_d) {
        int d = t - (RA_TS - 1);  // rl - ql
        T acc = 0;
        int lo = d > 0 ? d : 0, hi = d < 0 ? RA_TS + d : RA_TS;
        for (int i = lo; i < hi; ++i) acc += tile[(i - d) * (RA_TS + 1) + i];
        mypart[t] = acc;
      }
    } else if (t >= 128 && t < 128 + 2 * RA_TS - 1) {
      if (rel_a) {
        int sg = t - 128;  // rl + ql
        T acc = 0;
        int lo = sg - (RA_TS - 1) > 0 ? sg - (RA_TS - 1) : 0, hi = sg < RA_TS - 1 ? sg : RA_TS - 1;
        for (int i = lo; i <= hi; ++i) acc += tile[(sg - i) * (RA_TS + 1) + i];
        mypart[t] = acc;
      }
    }
  }
  if (!last_block_arrive(&counters[col], (unsigned)ntiles)) return;
  // ---- last block of this column: D_t for every tap t, fixed order ----
  const T* cp = part + (size_t)col * ntiles * RA_SLOTS;
  for (int t = threadIdx.x; t < s_red; t += blockDim.x) {
    double acc = 0.0;
    const int dl = t - c_red;  // global diagonal r - q
    // tiles (r0, q0) with |dl - (r0 - q0) TS| <= TS - 1, visited in a fixed order
    for (int delta = -(nt - 1); delta <= nt - 1; ++delta) {
      int dloc = dl - delta * RA_TS;
      if (dloc < -(RA_TS - 1) || dloc > RA_TS - 1) continue;
      for (int r0 = 0; r0 < nt; ++r0) {
        int q0 = r0 - delta;
        if (q0 < 0 || q0 >= nt) continue;
        acc += (double)__ldcg(cp + (size_t)(r0 + q0 * nt) * RA_SLOTS + dloc + RA_TS - 1);
      }
    }
    if (bc == KPSB_BC_REFLEXIVE) {
      for (int side = 0; side < 2; ++side) {
        int sg = side == 0 ? t - 1 - c_red : t - 1 - c_red + 2 * n;  // r + q
        if (sg < 0 || sg > 2 * n - 2) continue;
        int m_hi = sg / RA_TS, m_lo = m_hi - 1;
        for (int m = m_lo; m <= m_hi; ++m) {
          if (m < 0) continue;
          int sl = sg - m * RA_TS;
          if (sl < 0 || sl > 2 * RA_TS - 2) continue;
          for (int r0 = 0; r0 < nt; ++r0) {
            int q0 = m - r0;
            if (q0 < 0 || q0 >= nt) continue;
            acc += (double)__ldcg(cp + (size_t)(r0 + q0 * nt) * RA_SLOTS + 128 + sl);
          }
        }
      }
    }
    Dsh[t] = acc;
  }
  // the mix reads every PSF tap once per output: stage the PSF in shared memory (coalesced,
  // all threads) instead of one dependent global load per tap and output
  const int s1 = transpose ? s_red : s_exp;
  const bool staged = s0 * s1 <= MIX_N;
  if (staged)
    for (int e = threadIdx.x; e < s0 * s1; e += blockDim.x) Psh[e] = psf[e];
  __syncthreads();
  const T* P = staged ? Psh : psf;
  // mix: R: w_b = sum_a P(a,b) D_a ; R^T: w_a = sum_b P(a,b) D_b   (P column-major s0 x s1)
  for (int o = threadIdx.x; o < s_exp; o += blockDim.x) {
    double acc = 0.0;
    if (!transpose) {
      for (int a = 0; a < s_red; ++a) acc += (double)P[a + o * s0] * Dsh[a];
    } else {
      for (int b = 0; b < s_red; ++b) acc += (double)P[o + b * s0] * Dsh[b];
    }
    wout[(size_t)col * s_exp + o] = (T)acc;
  }
}

// U[i + j n] = sum over taps t with j = ext(i - t + c) of w_t, optionally + beta * prev.
template <typename T>
__global__ void __launch_bounds__(256) ra_expand_kernel(
    const T* __restrict__ wbuf, int s_exp, int c_exp, int n, int bc, T* __restrict__ U,
    int ldu, const T* __restrict__ prev, int ldp, const double* __restrict__ beta_dev,
    T beta_host, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ T w[RA_MAX_S];
  const int col = blockIdx.y;
  for (int t = threadIdx.x; t < s_exp; t += blockDim.x) w[t] = wbuf[(size_t)col * s_exp + t];
  __syncthreads();
  T beta = beta_dev ? (T)(*beta_dev) : beta_host;
  const long long N = (long long)n * n;
  T* u = U + (size_t)col * ldu;
  const T* pv = prev ? prev + (size_t)col * ldp : nullptr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e % n), j = (int)(e / n);
    T acc = 0;
    int t = i - j + c_exp;
    if (t >= 0 && t < s_exp) acc += w[t];
    if (bc == KPSB_BC_REFLEXIVE) {
      t = i + j + 1 + c_exp;
      if (t < s_exp) acc += w[t];
      t -= 2 * n;
      if (t >= 0 && t < s_exp) acc += w[t];
    }
    if (pv) acc = fma(beta, pv[e], acc);
    u[e] = acc;
  }
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

size_t ra_scratch_bytes(int n, int nb, int s_exp, size_t el) {
  int nt = (n + RA_TS - 1) / RA_TS;
  return align256((size_t)nb * sizeof(unsigned int)) + align256((size_t)nb * s_exp * el) +
         align256((size_t)nb * nt * nt * RA_SLOTS * el);
}

RAScratch ra_scratch_carve(void* base, int n, int nb, int s_exp, size_t el) {
  char* p = (char*)base;
  RAScratch s;
  s.counters = (unsigned int*)p;
  p += align256((size_t)nb * sizeof(unsigned int));
  s.w = (float*)p;
  p += align256((size_t)nb * s_exp * el);
  s.part = (float*)p;
  return s;
}

kpsb_status ra_check(int s0, int s1, int n, int bc) {
  KPSB_REQUIRE(n >= 2 && n <= KPSB_MAX_N, "n must be in [2, %d] (got %d)", KPSB_MAX_N, n);
  KPSB_REQUIRE(s0 >= 1 && s1 >= 1 && s0 <= RA_MAX_S && s1 <= RA_MAX_S,
               "PSF size %dx%d outside [1, %d]", s0, s1, RA_MAX_S);
  KPSB_REQUIRE(bc == KPSB_BC_ZERO || bc == KPSB_BC_REFLEXIVE, "unknown boundary condition %d", bc);
  if (bc == KPSB_BC_REFLEXIVE) {
    KPSB_REQUIRE(s0 / 2 <= n && s1 / 2 <= n && s0 - 1 - s0 / 2 <= n && s1 - 1 - s1 / 2 <= n,
                 "reflexive boundary needs the PSF overhang (%dx%d) within one image (%d)", s0,
                 s1, n);
  }
  return KPSB_OK;
}

template <typename T>
static kpsb_status ra_apply_t(const T* psf, int s0, int s1, int n, int bc, const T* V, int ldv, int nb, T* U,
                              int ldu, int transpose, const T* prev, int ldp, const double* beta_dev,
                              T beta_host, const int* skip, const RAScratch& scr, cudaStream_t st) {
  const int s_red = transpose ? s1 : s0, c_red = s_red / 2;
  const int s_exp = transpose ? s0 : s1, c_exp = s_exp / 2;
  const int nt = (n + RA_TS - 1) / RA_TS;
  dim3 g1(nt * nt, nb);
  ra_reduce_kernel<T><<<g1, 256, 0, st>>>(V, ldv, n, bc, s_red, c_red, s_exp, psf, s0, transpose,
                                          (T*)scr.part, scr.counters, (T*)scr.w);
  KPSB_CHECK_LAUNCH();
  long long N = (long long)n * n;
  int bx = (int)std::min<long long>((N + 255) / 256, 1024);
  dim3 g2(bx, nb);
  ra_expand_kernel<T><<<g2, 256, 0, st>>>((const T*)scr.w, s_exp, c_exp, n, bc, U, ldu, prev, ldp, beta_dev,
                                          beta_host, skip);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

kpsb_status ra_apply(const float* psf, int s0, int s1, int n, int bc, const float* V, int ldv,
                     int nb, float* U, int ldu, int transpose, const float* prev, int ldp,
                     const double* beta_dev, float beta_host, const int* skip,
                     const RAScratch& scr, cudaStream_t st) {
  return ra_apply_t<float>(psf, s0, s1, n, bc, V, ldv, nb, U, ldu, transpose, prev, ldp, beta_dev, beta_host,
                           skip, scr, st);
}

kpsb_status ra_apply(const double* psf, int s0, int s1, int n, int bc, const double* V, int ldv,
                     int nb, double* U, int ldu, int transpose, const double* prev, int ldp,
                     const double* beta_dev, double beta_host, const int* skip,
                     const RAScratch& scr, cudaStream_t st) {
  return ra_apply_t<double>(psf, s0, s1, n, bc, V, ldv, nb, U, ldu, transpose, prev, ldp, beta_dev,
                            beta_host, skip, scr, st);
}

// ---- dense R(A) from the index map (tests, explicit mode) -------------------------------
__global__ void ra_materialize_kernel(const float* __restrict__ psf, int s0, int s1, int n,
                                      int bc, float* __restrict__ R) {
  const long long N = (long long)n * n;
  const int c0 = s0 / 2, c1 = s1 / 2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N * N;
       e += (long long)gridDim.x * blockDim.x) {
    long long row = e % N, colx = e / N;
    int i = (int)(row % n), j = (int)(row / n);   // row (i, j): x-direction taps b
    int r = (int)(colx % n), q = (int)(colx / n); // column (r, q): y-direction taps a
    int bl[3], al[3], nbl = 0, nal = 0;
    int t = i - j + c1;
    if (t >= 0 && t < s1) bl[nbl++] = t;
    t = r - q + c0;
    if (t >= 0 && t < s0) al[nal++] = t;
    if (bc == KPSB_BC_REFLEXIVE) {
      t = i + j + 1 + c1;
      if (t < s1) bl[nbl++] = t;
      if (t - 2 * n >= 0 && t - 2 * n < s1) bl[nbl++] = t - 2 * n;
      t = r + q + 1 + c0;
      if (t < s0) al[nal++] = t;
      if (t - 2 * n >= 0 && t - 2 * n < s0) al[nal++] = t - 2 * n;
    }
    float acc = 0.f;
    for (int x = 0; x < nbl; ++x)
      for (int y = 0; y < nal; ++y) acc += psf[al[y] + bl[x] * s0];
    R[e] = acc;
  }
}

// ---- exact blur A and A^T (FP64) --------------------------------------------------------
__global__ void blur_kernel(const double* __restrict__ psf, int s0, int s1, int n, int bc,
                            const double* __restrict__ X, double* __restrict__ B, int transpose) {
  const long long N = (long long)n * n;
  const int c0 = s0 / 2, c1 = s1 / 2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
       e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e % n), c = (int)(e / n);
    double acc = 0.0;
    if (!transpose) {
      for (int b = 0; b < s1; ++b) {
        int cc = ext_index(c - b + c1, n, bc);
        if (cc < 0) continue;
        for (int a = 0; a < s0; ++a) {
          int rr = ext_index(r - a + c0, n, bc);
          if (rr < 0) continue;
          acc += psf[a + b * s0] * X[rr + (size_t)cc * n];
        }
      }
    } else {
      // A^T: output (r, c) gathers every (r', c') whose extended source is (r, c)
      for (int b = 0; b < s1; ++b) {
        int cand_c[3] = {c + b - c1, -1 - c + b - c1, 2 * n - 1 - c + b - c1};
        for (int xc = 0; xc < (bc == KPSB_BC_REFLEXIVE ? 3 : 1); ++xc) {
          int cp = cand_c[xc];
          if (cp < 0 || cp >= n || ext_index(cp - b + c1, n, bc) != c) continue;
          for (int a = 0; a < s0; ++a) {
            int cand_r[3] = {r + a - c0, -1 - r + a - c0, 2 * n - 1 - r + a - c0};
            for (int xr = 0; xr < (bc == KPSB_BC_REFLEXIVE ? 3 : 1); ++xr) {
              int rp = cand_r[xr];
              if (rp < 0 || rp >= n || ext_index(rp - a + c0, n, bc) != r) continue;
              acc += psf[a + b * s0] * X[rp + (size_t)cp * n];
            }
          }
        }
      }
    }
    B[e] = acc;
  }
}

}  // namespace kpsb

using namespace kpsb;

extern "C" kpsb_status kp_ra_apply_dev(const float* psf, int s0, int s1, int n, int bc,
                                       const float* V, int ldv, int nb, float* U, int ldu,
                                       int transpose, void* stream) {
  clear_error();
  KPSB_TRY(ra_check(s0, s1, n, bc));
  KPSB_REQUIRE(psf && V && U, "null pointer");
  KPSB_REQUIRE(nb >= 1 && ldv >= n * n && ldu >= n * n, "bad block shape nb=%d ldv=%d ldu=%d", nb,
               ldv, ldu);
  cudaStream_t st = (cudaStream_t)stream;
  const int s_exp = transpose ? s0 : s1;
  size_t bytes = ra_scratch_bytes(n, nb, s_exp);
  void* buf = nullptr;
  KPSB_TRY_CUDA(cudaMallocAsync(&buf, bytes, st));
  RAScratch scr = ra_scratch_carve(buf, n, nb, s_exp);
  cudaError_t e = cudaMemsetAsync(scr.counters, 0, (size_t)nb * sizeof(unsigned int), st);
  kpsb_status s = KPSB_OK;
  if (e != cudaSuccess) {
    set_error("cudaMemsetAsync: %s", cudaGetErrorString(e));
    s = KPSB_ECUDA;
  } else {
    s = ra_apply(psf, s0, s1, n, bc, V, ldv, nb, U, ldu, transpose, nullptr, 0, nullptr, 0.f,
                 nullptr, scr, st);
  }
  cudaFreeAsync(buf, st);
  return s;
}

extern "C" kpsb_status kp_ra_materialize_dev(const float* psf, int s0, int s1, int n, int bc,
                                             float* R, void* stream) {
  clear_error();
  KPSB_TRY(ra_check(s0, s1, n, bc));
  KPSB_REQUIRE(n <= 128, "materialised R(A) limited to n <= 128 (got %d)", n);
  KPSB_REQUIRE(psf && R, "null pointer");
  ra_materialize_kernel<<<152 * 8, 256, 0, (cudaStream_t)stream>>>(psf, s0, s1, n, bc, R);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

extern "C" kpsb_status kp_blur_dev(const double* psf, int s0, int s1, int n, int bc,
                                   const double* X, double* B, int transpose, void* stream) {
  clear_error();
  KPSB_TRY(ra_check(s0, s1, n, bc));
  KPSB_REQUIRE(psf && X && B && X != B, "null or aliased pointer");
  long long N = (long long)n * n;
  int blocks = (int)std::min<long long>((N + 255) / 256, 152 * 16);
  blur_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(psf, s0, s1, n, bc, X, B, transpose);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

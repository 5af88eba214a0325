// Split Bregman TV deblurring (Alg. 3 anisotropic, Alg. 4 isotropic) with CGLS (Alg. 5)
// on the augmented system Ahat = [sqrt(mu) A_k; lambda (L (x) I); lambda (I (x) L)]
// (eqs. (3.14)-(3.15)), batched over independent problems of one image size.
//
// FP64 vectors.  Per CGLS step: z1 = A_k w (KP GEMMs), |z|^2, x/r updates, f1 = A_k^T r1
// (KP GEMMs), f and |f|^2, w = f + delta w.  All scalars live on the device; every
// reduction is a fixed-order two-level sum, so results do not depend on the batch.
// L = 1/2 forward difference with a zero last row (Sec. 5.3): Dx acts along columns
// (horizontal, L_x (x) I), Dy along rows (vertical, I (x) L_y).
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <mutex>
#include <string>
#include <thread>

#include <cuda_bf16.h>

#include "fpconv.cuh"
#include "kpsb_internal.cuh"

namespace kpsb {

static constexpr int SB_T = 256;
// Minimum resident blocks per SM requested from the compiler for the vector kernels
// (register cap 65536 / (SB_T * blocks)).  They wait on memory latency, so more resident warps
// pay: the tensor-core path's kernels run 8 blocks (32 registers, a few bytes of spill; on the
// 256-request step 108.1 deblurs/s against 106.0 with 6 blocks, x update 684 -> 575 ms); the
// FP64 / FP32 path's kernels keep 6 (at 32 registers their spills grow to 48-80 bytes).
#ifndef KPSB_SB_MIN_BLOCKS
#define KPSB_SB_MIN_BLOCKS 6
#endif
#define SB_BOUNDS __launch_bounds__(SB_T, KPSB_SB_MIN_BLOCKS)
#ifndef KPSB_SB_MIN_BLOCKS_TC
#define KPSB_SB_MIN_BLOCKS_TC 8
#endif
#define SB_BOUNDS_TC __launch_bounds__(SB_T, KPSB_SB_MIN_BLOCKS_TC)
#ifndef KPSB_SB_MIN_BLOCKS_X
#define KPSB_SB_MIN_BLOCKS_X 8
#endif
#define SB_BOUNDS_X __launch_bounds__(SB_T, KPSB_SB_MIN_BLOCKS_X)  // x and r update kernels
// once-per-outer-step kernels and the CUDA-core path's x update, which would spill under
// the caps above
#define SB_BOUNDS_WIDE __launch_bounds__(SB_T, 4)
// Each block of a vector kernel handles one fixed chunk of SB_CHUNK elements (SB_EPT per
// thread) and writes one reduction partial: the summation order depends on n only, so a
// problem gives the same bits alone, in any batch, and in the serving loop.
#ifndef KPSB_SB_EPT
#define KPSB_SB_EPT 8
#endif
static constexpr int SB_EPT = KPSB_SB_EPT;  // 4, 8 or 16 (8: twice the blocks of 16, which
                                            // the concurrent parts interleave better)
static constexpr int SB_CHUNK = SB_T * SB_EPT;
static constexpr int SB_TILES_PER_CHUNK = SB_CHUNK / 1024;  // 32 x 32 tiles

struct SBScal {
  double tau;      // ||f||^2 of the current direction
  double step;     // mu_iota = tau / ||z||^2
  double delta;    // tau_{iota+1} / tau_iota
  double rc_cgls;
  double rc_sb;
  double ww;       // ||w||^2 of the current direction (tensor-core path: from the w kernel)
  double c1, c2;   // tensor-core path: -step sqrt(mu), -step lambda/2 (the x update's coefficients)
  int active;      // CGLS of the current outer step still running
  int sb_active;   // outer loop still running
  int it;          // CGLS steps in the current outer step
  int iota_total;
  int l_end;
  int pad;
};

#define dx_at tv_dx
#define dy_at tv_dy

__host__ __device__ __forceinline__ int sb_blocks(int n) {
  return (int)(((long long)n * n + SB_CHUNK - 1) / SB_CHUNK);
}

// Two-value fixed-order grid reduction inside one problem; returns true in the last block
// with the totals in out[0..1].
__device__ __forceinline__ bool prob_reduce2(const SBProb& P, double a, double b, double* out) {
  // block totals: partials through shared memory, added by one warp in a fixed order
  // (far fewer FP64 instructions than a shuffle tree in every warp)
  __shared__ double sa[SB_T], sb[SB_T];
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x < 32) {
    double ta = 0.0, tb = 0.0;
#pragma unroll
    for (int i = 0; i < SB_T / 32; ++i) {
      ta += sa[threadIdx.x + 32 * i];
      tb += sb[threadIdx.x + 32 * i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ta += __shfl_down_sync(0xffffffffu, ta, o);
      tb += __shfl_down_sync(0xffffffffu, tb, o);
    }
    if (threadIdx.x == 0) {
      P.part[2 * blockIdx.x] = ta;
      P.part[2 * blockIdx.x + 1] = tb;
    }
  }
  const unsigned nb = (unsigned)sb_blocks(P.n);
  if (!last_block_arrive(P.counter, nb)) return false;
  // the last block sums the partials in an order fixed by n alone: one warp up to 32 chunks
  // (n <= 256; no block barrier on this short path), the whole block above
  if (nb <= 32) {
    if (threadIdx.x < 32) {
      const double ta = warp_sum_strided(P.part, 2, (int)nb);
      const double tb = warp_sum_strided(P.part + 1, 2, (int)nb);
      if (threadIdx.x == 0) {
        out[0] = ta;
        out[1] = tb;
      }
    }
    return true;
  }
  const double ta = block_sum_strided(P.part, 2, (int)nb, sa);
  const double tb = block_sum_strided(P.part + 1, 2, (int)nb, sa);
  if (threadIdx.x == 0) {
    out[0] = ta;
    out[1] = tb;
  }
  return true;
}

// The same for one value (the kernels whose second total would be zero): half the FP64
// additions of the block and final sums.
__device__ __forceinline__ bool prob_reduce1(const SBProb& P, double a, double* out) {
  __shared__ double sa[SB_T];
  sa[threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    double ta = 0.0;
#pragma unroll
    for (int i = 0; i < SB_T / 32; ++i) ta += sa[threadIdx.x + 32 * i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ta += __shfl_down_sync(0xffffffffu, ta, o);
    if (threadIdx.x == 0) P.part[2 * blockIdx.x] = ta;
  }
  const unsigned nb = (unsigned)sb_blocks(P.n);
  if (!last_block_arrive(P.counter, nb)) return false;
  if (nb <= 32) {
    if (threadIdx.x < 32) {
      const double ta = warp_sum_strided(P.part, 2, (int)nb);
      if (threadIdx.x == 0) out[0] = ta;
    }
    return true;
  }
  const double ta = block_sum_strided(P.part, 2, (int)nb, sa);
  if (threadIdx.x == 0) out[0] = ta;
  return true;
}

#ifdef KPSB_SB_PROB_REF
#define SB_PROB_DECL const SBProb& P = probs[blockIdx.y];
#else
#define SB_PROB_DECL const SBProb P = probs[blockIdx.y];
#endif
#define SB_PROLOGUE(cond)                                            \
  SB_PROB_DECL                                                       \
  if ((int)blockIdx.x >= sb_blocks(P.n)) return;                     \
  if (!(cond)) return;                                               \
  const int n = P.n;                                                 \
  const long long N = (long long)n * n;                              \
  const long long e_lo = (long long)blockIdx.x * SB_CHUNK;           \
  const long long e_hi = e_lo + SB_CHUNK < N ? e_lo + SB_CHUNK : N;
// The elements of this block's chunk, SB_T apart.
#define SB_FOR_E for (long long e = e_lo + threadIdx.x; e < e_hi; e += SB_T)
// The same with the element's row r_ and column c_, advanced without a division per
// element (n * n < 2^32; r_ + SB_T % n < 2 n, so one wrap suffices).
#define SB_FOR_RC                                                                        \
  const unsigned e0_ = (unsigned)(e_lo + threadIdx.x), un_ = (unsigned)n;                \
  int r_ = (int)(e0_ % un_), c_ = (int)(e0_ / un_);                                      \
  const int dr_ = SB_T % n, dc_ = SB_T / n;                                              \
  for (long long e = e0_; e < e_hi;                                                      \
       e += SB_T, r_ += dr_, c_ += dc_, r_ >= n ? (r_ -= n, ++c_) : 0)

// x^(0) = b, d = g = 0, flags set (Alg. 3/4 initialisation).
__global__ void SB_BOUNDS sb_setup_kernel(const SBProb* __restrict__ probs) {
  SB_PROLOGUE(true)
  SB_FOR_E {
    P.x[e] = P.b[e];
    P.dx[e] = P.dy[e] = P.gx[e] = P.gy[e] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    memset(P.sc, 0, sizeof(SBScal));
    P.sc->sb_active = 1;
  }
}

// Outer step start: xprev = x; CGLS from x = 0 with r = bhat = [sqrt(mu) b; lam(dx-gx); lam(dy-gy)].
__global__ void SB_BOUNDS_WIDE sb_outer_init_kernel(const SBProb* __restrict__ probs) {
  SB_PROLOGUE(P.sc->sb_active)
  SB_FOR_E {
    P.xprev[e] = P.x[e];
    P.x[e] = 0.0;
    P.r1[e] = P.sqrt_mu * P.b[e];
    P.r2[e] = P.lam * (P.dx[e] - P.gx[e]);
    P.r3[e] = P.lam * (P.dy[e] - P.gy[e]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.sc->active = 1;
    P.sc->it = 0;
  }
}

// tau' = ||f||^2 (step 8), delta = tau'/tau (step 9); init: tau = tau', delta = 0.
__device__ __forceinline__ void f_scalars(SBScal* s, double taun, int init) {
  s->delta = init ? 0.0 : (s->tau > 0.0 ? taun / s->tau : 0.0);
  s->tau = taun;
  if (!(taun > 0.0)) s->active = 0;  // exact solution reached (or b-hat = 0)
}

// f = Ahat^T r = sqrt(mu) f1 + lam Dx^T r2 + lam Dy^T r3 (Alg. 5 step 7 / init) and
// tau' = ||f||^2 (step 8); delta = tau'/tau (step 9).  init: tau = tau', delta = 0.
__global__ void SB_BOUNDS sb_cgls_f_kernel(const SBProb* __restrict__ probs, int init) {
  SB_PROLOGUE(P.sc->active)
  // Dx^T r2 + Dy^T r3 = (lambda/2) t with t the raw differences (L = half forward difference,
  // zero last row); one coefficient per term keeps the FP64 operation count low.
  const double hl = 0.5 * P.lam;
  const bool unit_mu = P.sqrt_mu == 1.0;  // mu = 1 (every workload here): 1 * f1 is f1, skip the product
  double ss = 0.0;
  SB_FOR_RC {
    const int r = r_, c = c_;
    const double f1 = P.f1f ? f2d_bits(P.f1f[e]) : P.f1[e];
    double t = (c < n - 1 ? P.r2[e] : 0.0) + (r < n - 1 ? P.r3[e] : 0.0);
    if (c >= 1) t -= P.r2[e - n];
    if (r >= 1) t -= P.r3[e - 1];
    const double v = fma(hl, t, unit_mu ? f1 : P.sqrt_mu * f1);
    P.f[e] = v;
    ss = fma(v, v, ss);
  }
  double tot[2];
  if (!prob_reduce2(P, ss, 0.0, tot)) return;
  if (threadIdx.x == 0) f_scalars(P.sc, tot[0], init);
}

// w = f + delta w (step 10); init: w = f (step 2).  The start does not read w, which holds
// no value yet: 0 * w would turn leftover non-finite bytes into NaN.
__global__ void SB_BOUNDS sb_cgls_w_kernel(const SBProb* __restrict__ probs, int init) {
  SB_PROLOGUE(P.sc->active)
  const double dl = P.sc->delta;
  SB_FOR_E
    P.w[e] = init ? P.f[e] : fma(dl, P.w[e], P.f[e]);
}

// ||z||^2 with z = Ahat w = [sqrt(mu) z1; lam Dx w; lam Dy w] (steps 3-4).
__global__ void SB_BOUNDS sb_cgls_zz_kernel(const SBProb* __restrict__ probs) {
  SB_PROLOGUE(P.sc->active)
  // |z|^2 = mu |z1|^2 + (lambda/2)^2 (|raw Dx w|^2 + |raw Dy w|^2), two sums.  z1 from the
  // tensor-core apply is FP32: its squares are summed in FP32 per thread (SB_EPT terms), the
  // partials in FP64.
  double sz = 0.0, sd = 0.0;
  float szf = 0.0f;
  SB_FOR_RC {
    const int r = r_, c = c_;
    if (P.z1f) {
      const float z = P.z1f[e];
      szf = fmaf(z, z, szf);
    } else {
      const double z = P.z1[e];
      sz = fma(z, z, sz);
    }
    const double w = P.w[e];
    if (c < n - 1) {
      const double d = w - P.w[e + n];
      sd = fma(d, d, sd);
    }
    if (r < n - 1) {
      const double d = w - P.w[e + 1];
      sd = fma(d, d, sd);
    }
  }
  double tot[2];
  if (!prob_reduce2(P, sz + (double)szf, sd, tot)) return;
  if (threadIdx.x == 0) {
    SBScal* s = P.sc;
    const double hl = 0.5 * P.lam;
    const double zz = fma(hl * hl, tot[1], P.mu * tot[0]);
    if (zz > 0.0) {
      s->step = s->tau / zz;
    } else {
      s->step = 0.0;
      s->active = 0;
    }
  }
}

// x += mu w; r -= mu z (steps 5-6); RC_CGLS = ||mu w|| / ||x|| (eq. (5.1)) and the stop test.
__global__ void SB_BOUNDS_WIDE sb_cgls_x_kernel(const SBProb* __restrict__ probs) {
  SB_PROLOGUE(P.sc->active)
  const double mu = P.sc->step;
  const double c1 = -mu * P.sqrt_mu, c2 = -mu * (0.5 * P.lam);  // r -= mu z, one FMA each
  double sx = 0.0, sw = 0.0;
  SB_FOR_RC {
    const int r = r_, c = c_;
    const double w = P.w[e];
    const double xn = fma(mu, w, P.x[e]);
    P.x[e] = xn;
    P.r1[e] = fma(c1, P.z1[e], P.r1[e]);
    if (c < n - 1) P.r2[e] = fma(c2, w - P.w[e + n], P.r2[e]);  // last column: Dx w = 0
    if (r < n - 1) P.r3[e] = fma(c2, w - P.w[e + 1], P.r3[e]);  // last row: Dy w = 0
    sx = fma(xn, xn, sx);
    sw = fma(w, w, sw);
  }
  double tot[2];
  if (!prob_reduce2(P, sx, sw, tot)) return;
  if (threadIdx.x == 0) {
    SBScal* s = P.sc;
    double xn = sqrt(tot[0]);
    s->rc_cgls = xn > 0.0 ? mu * sqrt(tot[1]) / xn : INFINITY;
    s->it += 1;
    s->iota_total += 1;
    if (s->it >= P.i_max || (!P.fixed_inner && s->rc_cgls < P.tau_cgls)) s->active = 0;
  }
}

// Shrinkage (3.10) / (3.13) and Bregman updates (3.8)-(3.9); RC_SB (5.2).
__global__ void SB_BOUNDS_WIDE sb_shrink_kernel(const SBProb* __restrict__ probs) {
  SB_PROLOGUE(P.sc->sb_active)
  double sd = 0.0, sp = 0.0;
  const double thr = P.thr;
  SB_FOR_RC {
    const int r = r_, c = c_;
    double cx = dx_at(P.x, r, c, n) + P.gx[e];
    double cy = dy_at(P.x, r, c, n) + P.gy[e];
    double dxv, dyv;
    if (P.iso) {
      double s = sqrt(cx * cx + cy * cy);
      double sc = s > 0.0 ? fmax(s - thr, 0.0) / s : 0.0;
      dxv = cx * sc;
      dyv = cy * sc;
    } else {
      dxv = copysign(fmax(fabs(cx) - thr, 0.0), cx);
      dyv = copysign(fmax(fabs(cy) - thr, 0.0), cy);
    }
    P.dx[e] = dxv;
    P.dy[e] = dyv;
    P.gx[e] = cx - dxv;
    P.gy[e] = cy - dyv;
    double dd = P.x[e] - P.xprev[e], xp = P.xprev[e];
    sd = fma(dd, dd, sd);
    sp = fma(xp, xp, sp);
  }
  double tot[2];
  if (!prob_reduce2(P, sd, sp, tot)) return;
  if (threadIdx.x == 0) {
    SBScal* s = P.sc;
    s->rc_sb = tot[1] > 0.0 ? sqrt(tot[0]) / sqrt(tot[1]) : INFINITY;
    s->l_end += 1;
    if (s->l_end >= P.iters || s->rc_sb < P.tau_sb) s->sb_active = 0;
  }
}


// ---- tensor-core variant of the CGLS vector steps ---------------------------------------------
// With the fused tensor-core KP apply the GEMM epilogues already produce z1 and the pieces
// of |z|^2 (forward) and f with |f|^2 (transpose).  The kernels below finish each step and
// write the split TF32 planes Xt (row-major, Xt[r][m] = X(r, m), hi then lo) of the next
// apply's input themselves, working on 32 x 32 tiles so both the column-major vectors and
// the transposed planes are written coalesced.
#define SB_TILES_BEGIN                                                              \
  const int tn = n >> 5, ntile = tn * tn;                                           \
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;                           \
  const int t_hi = min(ntile, ((int)blockIdx.x + 1) * SB_TILES_PER_CHUNK);          \
  for (int t = (int)blockIdx.x * SB_TILES_PER_CHUNK; t < t_hi; ++t) {              \
    const int tr = t % tn, tcol = t / tn;
#define SB_TILES_END }

// Store the tile held in th/tl (th[col][row] of the tile) as rows of the Xt planes: FP32
// words holding TF32 values, or BF16 (the tile then holds BF16 values, converted exactly).
__device__ __forceinline__ void store_xt_tile(float* __restrict__ xt, int n, int tr, int tcol,
                                              float (*th)[33], float (*tl)[33], int lx, int ly, bool bf) {
  __syncthreads();
  const size_t nn = (size_t)n * n;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = tr * 32 + ly + 8 * j, m = tcol * 32 + lx;
    if (bf) {
      __nv_bfloat16* xb = (__nv_bfloat16*)xt;
      xb[(size_t)r * n + m] = __float2bfloat16_rn(th[lx][ly + 8 * j]);
      xb[nn + (size_t)r * n + m] = __float2bfloat16_rn(tl[lx][ly + 8 * j]);
    } else {
      xt[(size_t)r * n + m] = th[lx][ly + 8 * j];
      xt[nn + (size_t)r * n + m] = tl[lx][ly + 8 * j];
    }
  }
  __syncthreads();
}

// Writes the TF32 hi / lo split of v into the tile; returns v rounded to FP32.
// KPSB_SPLIT_INT_ROUND 1 rounds v to FP32 on the integer pipes (same bits as the conversion
// instruction, which issues to the FP64 pipe); 0 uses the conversion instruction.
#ifndef KPSB_SPLIT_INT_ROUND
#define KPSB_SPLIT_INT_ROUND 1
#endif
// KPSB_X_INT_WIDEN 1: the x update widens the FP32 apply result on the integer pipes.
#ifndef KPSB_X_INT_WIDEN
#define KPSB_X_INT_WIDEN 1
#endif
// KPSB_X_NORM_F32 1: ||x||^2 of the stop test from the FP32 rounding of x, summed in FP32 per
// thread (integer-pipe rounding, one FP32 FMA instead of an FP64 FMA per element).
#ifndef KPSB_X_NORM_F32
#define KPSB_X_NORM_F32 1
#endif
// With bf the split is BF16 (hi = bf16(f), lo = bf16(f - hi), round to nearest even), the
// same split the two-stage kernel's own split applies, held exactly in the FP32 tile.
__device__ __forceinline__ float put_split(float (*th)[33], float (*tl)[33], int a, int b, double v,
                                           bool bf) {
  const float f = KPSB_SPLIT_INT_ROUND ? d2f_rn_bits(v) : (float)v;
  if (bf) {
    const float h = __bfloat162float(__float2bfloat16_rn(f));
    th[a][b] = h;
    tl[a][b] = __bfloat162float(__float2bfloat16_rn(f - h));
  } else {
    const float h = tf32_rna(f);
    th[a][b] = h;
    tl[a][b] = tf32_rna(f - h);
  }
  return f;
}

// Outer step start (as sb_outer_init_kernel) plus the split planes of r1 = sqrt(mu) b.  The
// tensor-core path keeps the TV rows r2, r3 of the residual only as q = 2 (Dx^T r2 + Dy^T r3)
// / lambda (the raw differences): they enter the iteration only through Ahat^T r (step 7).
__global__ void SB_BOUNDS_TC sb_outer_init_tc_kernel(const SBProb* __restrict__ probs) {
  SB_PROLOGUE(P.sc->sb_active)
  (void)N; (void)e_hi;
  __shared__ float th[32][33], tl[32][33];
  SB_TILES_BEGIN
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = tr * 32 + lx, c = tcol * 32 + ly + 8 * j;
    const size_t e = r + (size_t)c * n;
    P.xprev[e] = P.x[e];
    P.x[e] = 0.0;
    const double r1 = P.sqrt_mu * P.b[e];
    P.r1[e] = r1;
    // q = raw TV part of Ahat^T r for r2 = lam (dx - gx), r3 = lam (dy - gy):
    // [c < n-1] r2(e) + [r < n-1] r3(e) - [c >= 1] r2(e - n) - [r >= 1] r3(e - 1)
    double t = 0.0;
    if (c < n - 1) t += P.dx[e] - P.gx[e];
    if (r < n - 1) t += P.dy[e] - P.gy[e];
    if (c >= 1) t -= P.dx[e - n] - P.gx[e - n];
    if (r >= 1) t -= P.dy[e - 1] - P.gy[e - 1];
    P.q[e] = P.lam * t;
    put_split(th, tl, ly + 8 * j, lx, r1, P.xt_bf16);
  }
  store_xt_tile(P.xt, n, tr, tcol, th, tl, lx, ly, P.xt_bf16);
  SB_TILES_END
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.sc->active = 1;
    P.sc->it = 0;
  }
}

// w = f + delta w (step 10; delta from the f kernel), init: w = f (step 2, w not read), and
// the planes and the FP32 value w_f of w for the next forward apply and ||z||^2.
__global__ void SB_BOUNDS_TC sb_w_tc_kernel(const SBProb* __restrict__ probs, int init) {
  SB_PROLOGUE(P.sc->active)
  (void)N; (void)e_hi;
  __shared__ float th[32][33], tl[32][33];
  const double dl = P.sc->delta;
  float wwf = 0.0f;  // ||w||^2 for RC_CGLS, from the FP32 value split below (SB_EPT terms per thread)
  SB_TILES_BEGIN
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = tr * 32 + lx, c = tcol * 32 + ly + 8 * j;
    const size_t e = r + (size_t)c * n;
    const double w = init ? P.f[e] : fma(dl, P.w[e], P.f[e]);
    P.w[e] = w;
    const float wf = put_split(th, tl, ly + 8 * j, lx, w, P.xt_bf16);
    P.wf[e] = wf;
    wwf = fmaf(wf, wf, wwf);
  }
  store_xt_tile(P.xt, n, tr, tcol, th, tl, lx, ly, P.xt_bf16);
  SB_TILES_END
  double tot[1];
  if (!prob_reduce1(P, f2d_bits(wwf), tot)) return;
  if (threadIdx.x == 0) P.sc->ww = tot[0];
}

// f = Ahat^T r = sqrt(mu) f1 + (lambda/2) q (step 7 / init) on the tensor-core path, f1 the
// FP32 apply result widened on the integer pipes; tau' = ||f||^2 and delta (steps 8-9).
__global__ void SB_BOUNDS_TC sb_f_tc_kernel(const SBProb* __restrict__ probs, int init) {
  SB_PROLOGUE(P.sc->active)
  const double hl = P.half_lam;
  double ss = 0.0;
  if (P.sqrt_mu == 1.0) {  // mu = 1: f1 as it is (the branch outside the loop: no product per element)
    SB_FOR_E {
      const double v = fma(hl, P.q[e], f2d_bits(P.f1f[e]));
      P.f[e] = v;
      ss = fma(v, v, ss);
    }
  } else {
    const double smu = P.sqrt_mu;
    SB_FOR_E {
      const double v = fma(hl, P.q[e], smu * f2d_bits(P.f1f[e]));
      P.f[e] = v;
      ss = fma(v, v, ss);
    }
  }
  double tot[1];
  if (!prob_reduce1(P, ss, tot)) return;
  if (threadIdx.x == 0) f_scalars(P.sc, tot[0], init);
}

// ||z||^2 with z = Ahat w_f (steps 3-4) on the tensor-core path: w_f = fl32(w) is the vector
// the forward apply saw and z1 = A_k w_f its FP32 result, so both sums,
// |z|^2 = mu |z1|^2 + (lambda/2)^2 |raw D w_f|^2, are sums of squares of FP32 values: taken
// in FP32 per thread (SB_EPT elements), the partials in FP64.  No FP64 arithmetic per element.
__global__ void SB_BOUNDS_TC sb_zz_tc_kernel(const SBProb* __restrict__ probs) {
  SB_PROLOGUE(P.sc->active)
  float sz = 0.0f, sd = 0.0f;
  SB_FOR_RC {
    const int r = r_, c = c_;
    const float z = P.z1f[e];
    sz = fmaf(z, z, sz);
    const float w = P.wf[e];
    if (c < n - 1) {
      const float d = w - P.wf[e + n];
      sd = fmaf(d, d, sd);
    }
    if (r < n - 1) {
      const float d = w - P.wf[e + 1];
      sd = fmaf(d, d, sd);
    }
  }
  double tot[2];
  if (!prob_reduce2(P, f2d_bits(sz), f2d_bits(sd), tot)) return;
  if (threadIdx.x == 0) {
    SBScal* s = P.sc;
    const double hl = 0.5 * P.lam;
    const double zz = fma(hl * hl, tot[1], P.mu * tot[0]);
    if (zz > 0.0) {
      s->step = s->tau / zz;
    } else {
      s->step = 0.0;
      s->active = 0;
    }
    s->c1 = -s->step * P.sqrt_mu;  // once here, not in every thread of the x update
    s->c2 = -s->step * (0.5 * P.lam);
  }
}

// x += mu w, r -= mu z (steps 5-6, mu from the zz kernel); RC_CGLS (5.1) and the stop
// test; the planes of r1 for the transpose apply.
__global__ void SB_BOUNDS_X sb_x_tc_kernel(const SBProb* __restrict__ probs) {
  SB_PROLOGUE(P.sc->active)
  (void)N; (void)e_hi;
  __shared__ float th[32][33], tl[32][33];
  const double mu = P.sc->step;
  const double c1 = P.sc->c1, c2 = P.sc->c2;  // r -= mu z, one FMA each (from the zz kernel)
  // ||w||^2 for RC_CGLS comes from the w kernel (sc->ww)
#if KPSB_X_NORM_F32
  float sxf = 0.0f;
#else
  double sx = 0.0;
#endif
  SB_TILES_BEGIN
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = tr * 32 + lx, c = tcol * 32 + ly + 8 * j;
    const size_t e = r + (size_t)c * n;
    const double w = P.w[e];
    const double xn = fma(mu, w, P.x[e]);
    P.x[e] = xn;
#if KPSB_X_INT_WIDEN
    const double z1 = f2d_bits(P.z1f[e]);
#else
    const double z1 = (double)P.z1f[e];
#endif
    const double r1 = fma(c1, z1, P.r1[e]);
    P.r1[e] = r1;
    // r2, r3 -= mu lam (Dx w_f, Dy w_f), the TV rows of z = Ahat w_f (the data row moves with
    // z1 = A_k w_f above), moves q by c2 (raw D^T D w_f)(e) = c2 (cnt w_f(e) - the sum of its cnt
    // neighbours inside the image): evaluated in FP32 on the FP32 values of the direction,
    // widened exactly, one FP64 FMA
    const float wr = c < n - 1 ? P.wf[e + n] : 0.f, wd = r < n - 1 ? P.wf[e + 1] : 0.f;
    const float wl = c >= 1 ? P.wf[e - n] : 0.f, wu = r >= 1 ? P.wf[e - 1] : 0.f;
    const float nb = (wr + wd) + (wl + wu);
    // the neighbour count (2, 3 or 4 for n >= 2) as a float from its bit pattern
    const int cnt = (c < n - 1) + (r < n - 1) + (c >= 1) + (r >= 1);
    const float cf = __int_as_float(cnt == 4 ? 0x40800000 : cnt == 3 ? 0x40400000 : 0x40000000);
    P.q[e] = fma(c2, f2d_bits(fmaf(cf, P.wf[e], -nb)), P.q[e]);
#if KPSB_X_NORM_F32
    const float xf = d2f_rn_bits(xn);
    sxf = fmaf(xf, xf, sxf);
#else
    sx = fma(xn, xn, sx);
#endif
    put_split(th, tl, ly + 8 * j, lx, r1, P.xt_bf16);
  }
  store_xt_tile(P.xt, n, tr, tcol, th, tl, lx, ly, P.xt_bf16);
  SB_TILES_END
  double tot[2];
#if KPSB_X_NORM_F32
  if (!prob_reduce1(P, f2d_bits(sxf), tot)) return;
#else
  if (!prob_reduce1(P, sx, tot)) return;
#endif
  if (threadIdx.x == 0) {
    SBScal* s = P.sc;
    const double xn = sqrt(tot[0]);
    s->rc_cgls = xn > 0.0 ? mu * sqrt(s->ww) / xn : INFINITY;
    s->it += 1;
    s->iota_total += 1;
    if (s->it >= P.i_max || (!P.fixed_inner && s->rc_cgls < P.tau_cgls)) s->active = 0;
  }
}

// Condition of the device-side CGLS loop (a WHILE node of the solve's CUDA graph): keep
// iterating while any problem of the batch is still active.  The per-node counter bounds
// the loop at `limit` iterations whatever the flags say.
__global__ void sb_cond_kernel(cudaGraphConditionalHandle h, const SBProb* __restrict__ probs, int P,
                               int* __restrict__ counter, int limit, int reset) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x)
    if (probs[p].sc->active) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = reset ? 0 : counter[0] + 1;
    counter[0] = c;
    if (!reset) counter[1] += 1;
    cudaGraphSetConditional(h, (any && c < limit) ? 1u : 0u);
  }
}

// Start gate of the parts that one batched call runs concurrently (one host thread each).
// Measured on GB300: a graph instantiation issued while other parts' graphs are running can
// wait for those graphs to finish (seconds) the first time a process holds that many live
// graphs; with every part's graph instantiated before any part launches, it never waits.
// A part arrives once: after instantiating its graph, or when it leaves without one.  The
// wait is bounded, so a part that never arrives costs the others at most that bound.
struct LaunchGate {
  std::mutex m;
  std::condition_variable cv;
  int arrived = 0, total = 0;
};
static thread_local LaunchGate* t_gate = nullptr;
static thread_local bool t_gate_done = false;

static void gate_arrive(bool wait) {
  LaunchGate* g = t_gate;
  if (!g || t_gate_done) return;
  t_gate_done = true;
  std::unique_lock<std::mutex> lk(g->m);
  if (++g->arrived >= g->total) {
    g->cv.notify_all();
  } else if (wait) {
    g->cv.wait_for(lk, std::chrono::seconds(30), [g] { return g->arrived >= g->total; });
  }
}

// Builds and runs `max_iters` outer steps of a batch as one CUDA graph: per outer step the
// head launches, a WHILE node whose body is one CGLS iteration plus the condition kernel,
// and the shrinkage (initialisation of new problems happens before, in sb_advance).  The graph is captured from the same launch sequences as the
// host-driven path.  Kernels that run inside the graph are counted after it completes.
template <class FHead, class FIter, class FShrink>
static kpsb_status sb_graph_run(cudaStream_t st, dim3 gv, const SBProb* dprobs, int P, int max_iters,
                                int i_max, int* ctrs, FHead& head, FIter& iter, FShrink& shrink,
                                int head_launches, int iter_launches) {
  cudaStream_t cs = nullptr, cs2 = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  kpsb_status s = KPSB_OK;
  cudaError_t e = cudaSuccess;
  bool capturing = false;
  set_capture_mode(true);
  do {
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking)) != cudaSuccess) break;
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) break;
    if ((e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
      break;
    capturing = true;
    for (int ell = 0; ell < max_iters; ++ell) {
      if ((s = head(cs))) break;
      cudaGraphConditionalHandle h;
      if ((e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) break;
      sb_cond_kernel<<<1, 256, 0, cs>>>(h, dprobs, P, ctrs, i_max + 2, 1);
      if ((e = cudaGetLastError()) != cudaSuccess) break;
      cudaStreamCaptureStatus cst;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      cudaGraph_t capg = nullptr;
      if ((e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, nullptr, &nd)) != cudaSuccess) break;
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t wn;
      if ((e = cudaGraphAddNode(&wn, capg, deps, nullptr, nd, &np)) != cudaSuccess) break;
      cudaGraph_t body = np.conditional.phGraph_out[0];
      if ((e = cudaStreamUpdateCaptureDependencies(cs, &wn, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
          cudaSuccess)
        break;
      if ((e = cudaStreamBeginCaptureToGraph(cs2, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        break;
      kpsb_status si = iter(cs2);
      if (si == KPSB_OK) {
        sb_cond_kernel<<<1, 256, 0, cs2>>>(h, dprobs, P, ctrs, i_max + 2, 0);
        e = cudaGetLastError();
      }
      cudaGraph_t body_out = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(cs2, &body_out);
      if (si) { s = si; break; }
      if (e == cudaSuccess) e = e2;
      if (e != cudaSuccess) break;
      if ((s = shrink(cs))) break;
    }
    cudaGraph_t gout = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &gout);
    capturing = false;
    if (s != KPSB_OK || e != cudaSuccess) break;
    if ((e = e2) != cudaSuccess) break;
    trace(st, "graph captured");
    if ((e = cudaGraphInstantiate(&ge, g, 0)) != cudaSuccess) break;
    if ((e = cudaGraphUpload(ge, st)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
    trace(st, "graph instantiated and uploaded");
    gate_arrive(true);
    trace(st, "graph launch");
    if ((e = cudaGraphLaunch(ge, st)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) break;
    trace(st, "graph done");
  } while (0);
  if (capturing) {
    cudaGraph_t tmp = nullptr;
    cudaStreamEndCapture(cs, &tmp);
  }
  set_capture_mode(false);
  if (s == KPSB_OK && e == cudaSuccess) {
    int h[2] = {0, 0};
    e = cudaMemcpy(h, ctrs, sizeof(h), cudaMemcpyDeviceToHost);
    // kernels executed: per outer step head + condition + shrink, per body run one CGLS
    // iteration + condition
    count_launch((long long)max_iters * (head_launches + 2) + (long long)h[1] * (iter_launches + 1));
  }
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  if (cs) cudaStreamDestroy(cs);
  if (cs2) cudaStreamDestroy(cs2);
  if (s == KPSB_OK && e != cudaSuccess) {
    set_error("split Bregman graph: %s", cudaGetErrorString(e));
    s = KPSB_ECUDA;
  }
  return s;
}

// ---- host driver -------------------------------------------------------------------------------
static size_t a256(size_t x) { return (x + 255) / 256 * 256; }

// GEMM arithmetic actually used for a size: tensor cores where the kernel tiles n, else
// FP32 (or FP64) CUDA cores.
static int gemm_prec_for(int n, int prec) {
  if (tc_supported(n, prec)) return prec;
  return prec == KPSB_P_FP64 ? KPSB_P_FP64 : KPSB_P_FP32;
}

// FP64 n^2 vectors of a problem's state: xprev, w, f, r1, r2, r3, z1, f1, dx, dy, gx, gy
// (b and x are the caller's)
static constexpr int SB_NVEC = 12;

size_t sb_state_bytes(int n, int k, int prec) {
  const size_t N = (size_t)n * n;
  const int gp = gemm_prec_for(n, prec);
  const size_t zbytes = tc_supported(n, gp) ? 0 : a256(kp_z_bytes(n, k, gp));
  size_t tc_ws = tc_supported(n, gp) ? a256(tc_plan_ws_bytes(n, k, gp)) : 0;
  return a256(SB_NVEC * N * sizeof(double)) + zbytes + a256(sizeof(SBScal)) +
         a256(sizeof(double) * sb_blocks(n) * 2) + 256 + tc_ws + a256(sizeof(float) * 5 * N) + 256;
}

kpsb_status sb_state_init(SBState* S, kpsb_kp* kp, const double* b_dev, double* x_dev, double mu,
                          double lambda, double beta, int tv, int iters, const kpsb_sb_opts& o,
                          cudaStream_t st) {
  const int n = kp->n;
  const size_t N = (size_t)n * n;
  S->kp = kp;
  S->n = n;
  S->prec = o.prec;
  const bool dense = kp->A_dense != nullptr;  // explicit A: FP64 products, partial-sum scratch
  S->gemm_prec = dense ? KPSB_P_FP64 : gemm_prec_for(n, o.prec);
  S->initialized = false;
  const size_t zbytes = dense ? a256(sizeof(double) * dense_partials(n))
                              : tc_supported(n, S->gemm_prec) ? 0 : a256(kp_z_bytes(n, kp->k, S->gemm_prec));
  // tensor-core applies with the split planes written by the vector kernels (32 x 32 tiles)
  // and FP32 results: any tensor-core precision, n a multiple of 32
  const bool fused = !dense && tc_supported(n, S->gemm_prec) && n % 32 == 0;
  const size_t xtbytes = fused ? a256(sizeof(float) * 5 * N) : 0;  // Xt planes + z1f + f1f + wf
  S->bytes = a256(SB_NVEC * N * sizeof(double)) + zbytes + a256(sizeof(SBScal)) +
             a256(sizeof(double) * sb_blocks(n) * 2) + 256 + xtbytes;
  KPSB_TRY_CUDA(cudaMallocAsync((void**)&S->mem, S->bytes, st));
  char* q = S->mem;
  double* v = (double*)q;
  SBProb& P = S->prob;
  P.n = n;
  P.iters = iters;
  P.iso = tv == KPSB_ISO;
  P.fixed_inner = o.fixed_inner;
  P.i_max = o.i_max;
  P.mu = mu;
  P.sqrt_mu = sqrt(mu);
  P.lam = lambda;
  P.half_lam = 0.5 * lambda;
  P.thr = o.threshold_rule == KPSB_THR_PAPER ? beta / (lambda * lambda) : beta / (2.0 * lambda * lambda);
  P.tau_cgls = o.tau_cgls;
  P.tau_sb = o.tau_sb;
  P.b = b_dev;
  P.x = x_dev;
  P.xprev = v + 0 * N; P.w = v + 1 * N; P.f = v + 2 * N; P.r1 = v + 3 * N; P.r2 = v + 4 * N;
  P.r3 = v + 5 * N; P.z1 = v + 6 * N; P.f1 = v + 7 * N; P.dx = v + 8 * N; P.dy = v + 9 * N;
  P.gx = v + 10 * N; P.gy = v + 11 * N;
  P.q = P.r2;  // the tensor-core path keeps q where the other paths keep r2 (and no r3)
  q += a256(SB_NVEC * N * sizeof(double));
  S->Z = zbytes ? (void*)q : nullptr;
  q += zbytes;
  P.sc = (SBScal*)q;
  q += a256(sizeof(SBScal));
  P.part = (double*)q;
  q += a256(sizeof(double) * sb_blocks(n) * 2);
  P.counter = (unsigned int*)q;
  q += 256;
  P.xt = fused ? (float*)q : nullptr;
  P.xt_bf16 = S->gemm_prec == KPSB_P_BF16X3 || S->gemm_prec == KPSB_P_BF16X2;
  P.z1f = fused ? P.xt + 2 * N : nullptr;
  P.f1f = fused ? P.xt + 3 * N : nullptr;
  P.wf = fused ? P.xt + 4 * N : nullptr;
  // the block comes from the stream-ordered pool with whatever its last user left: clear it
  // all, so that no read of a not-yet-written vector can depend on that history
  KPSB_TRY_CUDA(cudaMemsetAsync(S->mem, 0, S->bytes, st));
  return KPSB_OK;
}

void sb_state_free(SBState* S, cudaStream_t st) {
  if (S && S->mem) {
    cudaFreeAsync(S->mem, st);
    S->mem = nullptr;
  }
}

kpsb_status sb_state_read(SBState* const* set, int count, std::vector<kpsb_sb_stats>& out,
                          std::vector<int>& done, cudaStream_t st) {
  SBScal* hsc = nullptr;
  KPSB_TRY_CUDA(cudaMallocHost((void**)&hsc, sizeof(SBScal) * std::max(1, count)));
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < count && e == cudaSuccess; ++p)
    e = cudaMemcpyAsync(hsc + p, set[p]->prob.sc, sizeof(SBScal), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    out.resize(count);
    done.resize(count);
    for (int p = 0; p < count; ++p) {
      out[p].l_end = hsc[p].l_end;
      out[p].iota_total = hsc[p].iota_total;
      out[p].rc_sb = hsc[p].rc_sb;
      out[p].status = KPSB_OK;
      done[p] = set[p]->initialized && !hsc[p].sb_active;
    }
  }
  cudaFreeHost(hsc);
  if (e != cudaSuccess) {
    set_error("reading split Bregman state: %s", cudaGetErrorString(e));
    return KPSB_ECUDA;
  }
  return KPSB_OK;
}

// Advances every state of `set` (all with the same n) by up to `outer_steps` outer split
// Bregman steps: states not yet initialised get x = b, d = g = 0 first; finished states
// do nothing.  Production runs one CUDA graph; with GEMM timing on, a host-driven loop.
kpsb_status sb_advance(SBState* const* set, int count, int outer_steps, const kpsb_sb_opts& o,
                       cudaStream_t st) {
  if (count <= 0 || outer_steps <= 0) return KPSB_OK;
  const int P = count;
  const int n = set[0]->n;
  int kmax = 0;
  for (int p = 0; p < P; ++p) kmax = std::max(kmax, set[p]->kp->k);
  const bool dense = set[0]->kp->A_dense != nullptr;  // a group is all explicit or all KP
  const int gemm_prec = dense ? KPSB_P_FP64 : gemm_prec_for(n, o.prec);
  const bool tc = !dense && tc_supported(n, gemm_prec);
  // fused CGLS variant: every state carries split planes and epilogue partials
  bool fz = tc && n % 32 == 0;
  for (int p = 0; p < count; ++p) fz = fz && set[p]->prob.xt != nullptr;
  const size_t small = a256(sizeof(SBProb) * P) * 2 + 2 * a256(sizeof(KPJob) * P) + 256;
  char* base = nullptr;
  KPSB_TRY_CUDA(cudaMallocAsync((void**)&base, small, st));
  std::vector<SBProb> hp(P), hnew;
  std::vector<KPJob> fwd(P), bwd(P);
  std::vector<kpsb_kp*> kps(P);
  for (int p = 0; p < P; ++p) {
    const SBState* S = set[p];
    hp[p] = S->prob;
    if (!S->initialized) hnew.push_back(S->prob);
    kps[p] = S->kp;
    KPJob& F = fwd[p];
    F.Ax = S->kp->Ax; F.Ay = S->kp->Ay; F.sigma = S->kp->sigma_d; F.n = n; F.k = S->kp->k;
    F.X = S->prob.w; F.Y = S->prob.z1; F.Z = S->Z;
    F.A = S->kp->A_dense;
    F.active = (const int*)((char*)S->prob.sc + offsetof(SBScal, active));
    KPJob& B = bwd[p];
    B = F;
    B.X = S->prob.r1; B.Y = S->prob.f1;
    if (fz) {  // fused kernel: inputs split by the vector kernels, FP32 results
      F.xt_ext = B.xt_ext = S->prob.xt;
      F.yf = S->prob.z1f;
      B.yf = S->prob.f1f;
    }
  }
  SBProb* dprobs = (SBProb*)base;
  SBProb* dnew = (SBProb*)(base + a256(sizeof(SBProb) * P));
  KPJob* dfwd = (KPJob*)((char*)dnew + a256(sizeof(SBProb) * P));
  KPJob* dbwd = (KPJob*)((char*)dfwd + a256(sizeof(KPJob) * P));
  int* ctrs = (int*)((char*)dbwd + a256(sizeof(KPJob) * P));  // [0] loop counter, [1] body runs
  kpsb_status s = KPSB_OK;
  cudaError_t e = cudaSuccess;
  SBScal* hsc = nullptr;
  TCPlan* plan = nullptr;
  do {
    e = cudaMemcpyAsync(dprobs, hp.data(), sizeof(SBProb) * P, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !hnew.empty())
      e = cudaMemcpyAsync(dnew, hnew.data(), sizeof(SBProb) * hnew.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dfwd, fwd.data(), sizeof(KPJob) * P, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dbwd, bwd.data(), sizeof(KPJob) * P, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctrs, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&hsc, sizeof(SBScal) * P);
    if (e != cudaSuccess) { set_error("sb setup: %s", cudaGetErrorString(e)); s = KPSB_ECUDA; break; }
    const int blocks = sb_blocks(n);
    dim3 gv(blocks, P);
    if (!hnew.empty()) {
      sb_setup_kernel<<<dim3(blocks, (unsigned)hnew.size()), SB_T, 0, st>>>(dnew);
      KPSB_CHECK_LAUNCH();
      for (int p = 0; p < P; ++p) set[p]->initialized = true;
    }
    double ksum = 0.0;
    for (int p = 0; p < P; ++p) ksum += set[p]->kp->k;
    const double apply_flops = 4.0 * ksum * (double)n * n * n;  // 4 k n^3 per problem (Sec. 4.2)
    trace(st, "advance setup queued");
    // one of several concurrent parts of a batch: its applies share the SMs with the others
    const bool shared = t_gate && t_gate->total > 1;
    if (tc && (s = tc_plan_create(kps.data(), fwd.data(), bwd.data(), P, n, gemm_prec, st, &plan, shared))) break;
    trace(st, "apply plan ready");
    // kernel launches of one apply (forward / transpose)
    const int apply_launches = tc ? tc_plan_launches(plan) : 3;
    const int ap_f = dense ? 2 : apply_launches, ap_b = dense ? 1 : apply_launches;
    const bool timed = gemm_timing_enabled();
    // One KP apply of the whole batch on stream sx (timed with events in instrumented mode).
    auto kp_apply_on = [&](int transpose, cudaStream_t sx) -> kpsb_status {
      int slot = timed ? gemm_timer_begin(sx) : -1;
      kpsb_status r = dense ? dense_apply_batch(transpose ? dbwd : dfwd, P, n, transpose, sx)
                      : tc  ? tc_plan_apply(plan, transpose, sx)
                            : kp_apply_batch(transpose ? dbwd : dfwd, P, n, kmax, transpose, gemm_prec, sx);
      gemm_timer_end(slot, sx, apply_flops, transpose ? ap_b : ap_f);
      return r;
    };
    // Vector kernels: in the instrumented mode each launch is bracketed by an event pair
    // of its category.
#define SB_LAUNCH(cat, kernel, ...)                                    \
  do {                                                                 \
    const int slot_ = timed ? timer_begin(sx) : -1;                    \
    kernel<<<gv, SB_T, 0, sx>>>(__VA_ARGS__);                          \
    KPSB_CHECK_LAUNCH();                                               \
    timer_end(slot_, sx, cat, 0.0, 1);                                 \
  } while (0)
    // Head of an outer step: x_prev = x, CGLS start r = bhat, f = Ahat^T r, w = f.
    auto outer_head = [&](cudaStream_t sx) -> kpsb_status {
      if (fz) {
        SB_LAUNCH(TIMER_SB_OUTER, sb_outer_init_tc_kernel, dprobs);
        KPSB_TRY(kp_apply_on(1, sx));
        SB_LAUNCH(TIMER_SB_F, sb_f_tc_kernel, dprobs, 1);
        SB_LAUNCH(TIMER_SB_W, sb_w_tc_kernel, dprobs, 1);
        return KPSB_OK;
      }
      SB_LAUNCH(TIMER_SB_OUTER, sb_outer_init_kernel, dprobs);
      KPSB_TRY(kp_apply_on(1, sx));
      SB_LAUNCH(TIMER_SB_F, sb_cgls_f_kernel, dprobs, 1);
      SB_LAUNCH(TIMER_SB_W, sb_cgls_w_kernel, dprobs, 1);
      return KPSB_OK;
    };
    // One CGLS iteration (Alg. 5 steps 3-10) of every active problem.
    auto cgls_iter = [&](cudaStream_t sx) -> kpsb_status {
      if (fz) {
        KPSB_TRY(kp_apply_on(0, sx));
        SB_LAUNCH(TIMER_SB_ZZ, sb_zz_tc_kernel, dprobs);
        SB_LAUNCH(TIMER_SB_X, sb_x_tc_kernel, dprobs);
        KPSB_TRY(kp_apply_on(1, sx));
        SB_LAUNCH(TIMER_SB_F, sb_f_tc_kernel, dprobs, 0);
        SB_LAUNCH(TIMER_SB_W, sb_w_tc_kernel, dprobs, 0);
        return KPSB_OK;
      }
      KPSB_TRY(kp_apply_on(0, sx));
      SB_LAUNCH(TIMER_SB_ZZ, sb_cgls_zz_kernel, dprobs);
      SB_LAUNCH(TIMER_SB_X, sb_cgls_x_kernel, dprobs);
      KPSB_TRY(kp_apply_on(1, sx));
      SB_LAUNCH(TIMER_SB_F, sb_cgls_f_kernel, dprobs, 0);
      SB_LAUNCH(TIMER_SB_W, sb_cgls_w_kernel, dprobs, 0);
      return KPSB_OK;
    };
    auto shrink = [&](cudaStream_t sx) -> kpsb_status {
      SB_LAUNCH(TIMER_SB_OUTER, sb_shrink_kernel, dprobs);
      return KPSB_OK;
    };
#undef SB_LAUNCH
    if (!timed) {
      // Production path: the whole advance is one CUDA graph; each outer step's CGLS loop
      // is a device-side WHILE node, so no host round trip happens until the end.
      s = sb_graph_run(st, gv, dprobs, P, outer_steps, o.i_max, ctrs, outer_head, cgls_iter, shrink,
                       3 + ap_b, 4 + ap_f + ap_b);
      if (s) break;
    } else {
      // Instrumented path: host-driven loop (CUDA events around every KP apply), checking
      // the device flags every few CGLS iterations.
      gate_arrive(false);
      const int CHUNK = 4;
      for (int ell = 0; ell < outer_steps && s == KPSB_OK; ++ell) {
        if ((s = outer_head(st))) break;
        for (int it = 0; it < o.i_max; ++it) {
          if ((s = cgls_iter(st))) break;
          if (!o.fixed_inner && (it + 1) % CHUNK == 0 && it + 1 < o.i_max) {
            for (int p = 0; p < P && e == cudaSuccess; ++p)
              e = cudaMemcpyAsync(hsc + p, hp[p].sc, sizeof(SBScal), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) break;
            bool any = false;
            for (int p = 0; p < P; ++p) any |= hsc[p].active != 0;
            if (!any) break;
          }
        }
        if (s) break;
        if (e != cudaSuccess) { set_error("sb loop: %s", cudaGetErrorString(e)); s = KPSB_ECUDA; break; }
        if ((s = shrink(st))) break;
      }
      if (s) break;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { set_error("sb loop: %s", cudaGetErrorString(e)); s = KPSB_ECUDA; break; }
    }
    if (tc && (s = tc_check_error())) break;
  } while (0);
  if (hsc) cudaFreeHost(hsc);
  if (plan) tc_plan_free(plan, st);
  cudaFreeAsync(base, st);
  return s;
}

struct SBJobIn {
  kpsb_kp* kp;
  const double* b;  // device
  double* x;        // device
  double mu, lambda, beta;
  int tv, iters;
};

// Runs all jobs (same n) to completion on stream st.  stats_out receives one entry per job.
static kpsb_status sb_run_group(const std::vector<SBJobIn>& jobs, const kpsb_sb_opts& o,
                                cudaStream_t st, std::vector<kpsb_sb_stats>& stats_out) {
  const int P = (int)jobs.size();
  std::vector<SBState> states(P);
  std::vector<SBState*> set(P);
  kpsb_status s = KPSB_OK;
  int made = 0;
  for (; made < P && s == KPSB_OK; ++made) {
    const SBJobIn& J = jobs[made];
    s = sb_state_init(&states[made], J.kp, J.b, J.x, J.mu, J.lambda, J.beta, J.tv, J.iters, o, st);
    set[made] = &states[made];
  }
  int max_iters = 0;
  for (auto& j : jobs) max_iters = std::max(max_iters, j.iters);
  if (s == KPSB_OK) s = sb_advance(set.data(), P, max_iters, o, st);
  std::vector<int> done;
  if (s == KPSB_OK) s = sb_state_read(set.data(), P, stats_out, done, st);
  for (int p = 0; p < made; ++p) sb_state_free(&states[p], st);
  return s;
}

kpsb_status sb_fill_defaults(const kpsb_sb_opts* opts, kpsb_sb_opts& o) {
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.tau_cgls <= 0.0) o.tau_cgls = 1e-4;
  if (o.i_max <= 0) o.i_max = 100;
  KPSB_REQUIRE(o.sub_batches >= 0, "sub_batches must be >= 0 (got %d)", o.sub_batches);
  KPSB_REQUIRE(prec_valid(o.prec), "unknown precision %d", o.prec);
  KPSB_REQUIRE(o.threshold_rule == KPSB_THR_EXACT || o.threshold_rule == KPSB_THR_PAPER,
               "unknown threshold rule %d", o.threshold_rule);
  return KPSB_OK;
}

static kpsb_status sb_check_job(kpsb_kp* kp, double mu, double lambda, int tv, int iters) {
  KPSB_REQUIRE(kp, "null handle");
  KPSB_REQUIRE(mu > 0.0 && lambda > 0.0 && isfinite(mu) && isfinite(lambda), "mu and lambda must be > 0");
  KPSB_REQUIRE(tv == KPSB_ANISO || tv == KPSB_ISO, "unknown TV type %d", tv);
  KPSB_REQUIRE(iters >= 1, "iters must be >= 1");
  return KPSB_OK;
}

}  // namespace kpsb

using namespace kpsb;

extern "C" kpsb_status sb_solve_dev(kpsb_kp_t kp, const double* b, double mu, double lambda, int tv,
                                    int iters, const kpsb_sb_opts* opts, double* x_out,
                                    kpsb_sb_stats* stats) {
  clear_error();
  KPSB_TRY(sb_check_job(kp, mu, lambda, tv, iters));
  KPSB_REQUIRE(b && x_out && b != x_out, "null or aliased pointer");
  kpsb_sb_opts o;
  KPSB_TRY(sb_fill_defaults(opts, o));
  double beta = o.beta > 0.0 ? o.beta : lambda * lambda / 2.0;
  std::vector<SBJobIn> jobs(1);
  jobs[0] = SBJobIn{kp, b, x_out, mu, lambda, beta, tv, iters};
  std::vector<kpsb_sb_stats> st;
  kpsb_status s = sb_run_group(jobs, o, (cudaStream_t)o.stream, st);
  if (s == KPSB_OK && stats) *stats = st[0];
  return s;
}

extern "C" kpsb_status sb_solve(kpsb_kp_t kp, const double* b, double mu, double lambda, int tv,
                                int iters, const kpsb_sb_opts* opts, double* x_out,
                                kpsb_sb_stats* stats) {
  clear_error();
  KPSB_TRY(sb_check_job(kp, mu, lambda, tv, iters));
  KPSB_REQUIRE(b && x_out, "null pointer");
  const size_t bytes = sizeof(double) * (size_t)kp->n * kp->n;
  kpsb_sb_opts o;
  KPSB_TRY(sb_fill_defaults(opts, o));
  cudaStream_t st = (cudaStream_t)o.stream;
  double* d = nullptr;
  KPSB_TRY_CUDA(cudaMallocAsync((void**)&d, 2 * bytes, st));
  kpsb_status s = KPSB_OK;
  cudaError_t e = cudaMemcpyAsync(d, b, bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    s = sb_solve_dev(kp, d, mu, lambda, tv, iters, &o, d + bytes / sizeof(double), stats);
    if (s == KPSB_OK) e = cudaMemcpyAsync(x_out, d + bytes / sizeof(double), bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFreeAsync(d, st);
  if (e != cudaSuccess) {
    set_error("sb_solve: %s", cudaGetErrorString(e));
    return KPSB_ECUDA;
  }
  return s;
}

extern "C" kpsb_status sb_solve_batched(int count, const kpsb_sb_job* jobs, int on_device,
                                        const kpsb_sb_opts* opts) {
  clear_error();
  KPSB_REQUIRE(count >= 0 && (count == 0 || jobs), "bad batch");
  if (count == 0) return KPSB_OK;
  kpsb_sb_opts o;
  KPSB_TRY(sb_fill_defaults(opts, o));
  cudaStream_t st = (cudaStream_t)o.stream;
  for (int i = 0; i < count; ++i) {
    KPSB_TRY(sb_check_job(jobs[i].kp, jobs[i].mu, jobs[i].lambda, jobs[i].tv, jobs[i].iters));
    KPSB_REQUIRE(jobs[i].b && jobs[i].x, "job %d: null pointer", i);
  }
  // group by image size; each group shares its launches
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  // groups: same n and same operator kind (Kronecker sum or explicit A)
  auto gkey = [&](int i) { return 2LL * jobs[i].kp->n + (jobs[i].kp->A_dense ? 1 : 0); };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return gkey(a) < gkey(b); });
  size_t host_bytes = 0;
  for (int i = 0; i < count; ++i) host_bytes += 2 * sizeof(double) * (size_t)jobs[i].kp->n * jobs[i].kp->n;
  double* dbuf = nullptr;
  if (!on_device) KPSB_TRY_CUDA(cudaMallocAsync((void**)&dbuf, host_bytes, st));
  std::vector<double*> db(count), dx(count);
  kpsb_status s = KPSB_OK;
  cudaError_t e = cudaSuccess;
  size_t off = 0;
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    size_t nn = (size_t)jobs[i].kp->n * jobs[i].kp->n;
    if (on_device) {
      db[i] = const_cast<double*>(jobs[i].b);
      dx[i] = jobs[i].x;
    } else {
      db[i] = dbuf + off;
      dx[i] = dbuf + off + nn;
      off += 2 * nn;
      e = cudaMemcpyAsync(db[i], jobs[i].b, nn * sizeof(double), cudaMemcpyHostToDevice, st);
    }
  }
  if (e != cudaSuccess) {
    set_error("sb_solve_batched upload: %s", cudaGetErrorString(e));
    s = KPSB_ECUDA;
  }
  // groups [g0, g1) of the sorted order; a large group may be cut into parts that run
  // concurrently (each part is an independent batch: same per-problem arithmetic)
  std::vector<std::pair<int, int>> groups;
  for (int g0 = 0; g0 < count;) {
    int g1 = g0;
    while (g1 < count && gkey(order[g1]) == gkey(order[g0])) ++g1;
    const int size = g1 - g0;
    const int np = std::max(1, std::min(size, o.sub_batches > 0 ? o.sub_batches : std::min(4, size / 64)));
    for (int q = 0; q < np; ++q) groups.emplace_back(g0 + size * q / np, g0 + size * (q + 1) / np);
    g0 = g1;
  }
  std::vector<kpsb_status> gs(groups.size(), KPSB_OK);
  std::vector<std::string> gerr(groups.size());
  auto run_group = [&](size_t gi, cudaStream_t gst) {
    std::vector<SBJobIn> grp;
    for (int t = groups[gi].first; t < groups[gi].second; ++t) {
      const kpsb_sb_job& J = jobs[order[t]];
      double beta = J.beta > 0.0 ? J.beta : J.lambda * J.lambda / 2.0;
      grp.push_back(SBJobIn{J.kp, db[order[t]], dx[order[t]], J.mu, J.lambda, beta, J.tv, J.iters});
    }
    std::vector<kpsb_sb_stats> stv;
    gs[gi] = sb_run_group(grp, o, gst, stv);
    if (gs[gi] == KPSB_OK) {
      for (int t = groups[gi].first; t < groups[gi].second; ++t)
        if (jobs[order[t]].stats) *jobs[order[t]].stats = stv[t - groups[gi].first];
    } else {
      gerr[gi] = kpsb_last_error();
    }
  };
  if (s == KPSB_OK && groups.size() == 1) {
    run_group(0, st);
  } else if (s == KPSB_OK) {
    // Size groups are independent: each runs on its own stream from its own host thread,
    // so small latency-bound groups overlap the large ones.  Every group starts after the
    // uploads on st; the downloads below start after every group has synchronised.
    int dev = 0;
    cudaEvent_t up = nullptr;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&up, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(up, st);
    if (e != cudaSuccess) {
      set_error("sb_solve_batched: %s", cudaGetErrorString(e));
      s = KPSB_ECUDA;
    } else {
      std::vector<std::thread> th;
      LaunchGate gate;
      gate.total = (int)groups.size();
      for (size_t gi = 0; gi < groups.size(); ++gi)
        th.emplace_back([&, gi] {
          t_gate = &gate;
          t_gate_done = false;
          cudaStream_t gst = nullptr;
          cudaError_t ge = cudaSetDevice(dev);
          if (ge == cudaSuccess) ge = cudaStreamCreateWithFlags(&gst, cudaStreamNonBlocking);
          if (ge == cudaSuccess) ge = cudaStreamWaitEvent(gst, up, 0);
          if (ge == cudaSuccess) {
            run_group(gi, gst);
            ge = cudaStreamSynchronize(gst);
          }
          gate_arrive(false);  // a part that left before launching a graph
          t_gate = nullptr;
          if (gst) cudaStreamDestroy(gst);
          if (ge != cudaSuccess && gs[gi] == KPSB_OK) {
            gs[gi] = KPSB_ECUDA;
            gerr[gi] = std::string("size group stream: ") + cudaGetErrorString(ge);
          }
        });
      for (auto& t : th) t.join();
    }
    if (up) cudaEventDestroy(up);
  }
  for (size_t gi = 0; gi < groups.size() && s == KPSB_OK; ++gi)
    if (gs[gi] != KPSB_OK) {
      set_error("%s", gerr[gi].c_str());
      s = gs[gi];
    }
  if (s == KPSB_OK && !on_device) {
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
      size_t nn = (size_t)jobs[i].kp->n * jobs[i].kp->n;
      e = cudaMemcpyAsync(jobs[i].x, dx[i], nn * sizeof(double), cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      set_error("sb_solve_batched download: %s", cudaGetErrorString(e));
      s = KPSB_ECUDA;
    }
  }
  if (dbuf) cudaFreeAsync(dbuf, st);
  if (s == KPSB_OK) cudaStreamSynchronize(st);
  return s;
}

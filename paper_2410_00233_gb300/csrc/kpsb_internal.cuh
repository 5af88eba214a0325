// Internal declarations shared by the translation units of the kpsb library.
#pragma once

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace kpsb {

// ---- R(A) block apply (ra.cu) -----------------------------------------------------------
struct RAScratch {
  float* part;             // per-tile diagonal / anti-diagonal partial sums (element type of V)
  float* w;                // mixed tap weights, nb x s_exp (element type of V)
  unsigned int* counters;  // last-block counters, nb (must start at zero)
};
// el = sizeof the element type of the vectors (float or double)
size_t ra_scratch_bytes(int n, int nb, int s_exp, size_t el = sizeof(float));
RAScratch ra_scratch_carve(void* base, int n, int nb, int s_exp, size_t el = sizeof(float));
kpsb_status ra_check(int s0, int s1, int n, int bc);
// The same products for a general operator given as an explicit FP32 matrix A (N x N,
// column-major): R(A)[i + j n, p + q n] = A[(i n + p) + (j n + q) N] (ra_dense.cu).
kpsb_status ra_dense_apply(const float* A, int n, const float* V, int ldv, int nb, float* U, int ldu,
                           int transpose, const float* prev, int ldp, const double* beta_dev,
                           float beta_host, const int* skip, cudaStream_t st);
// U = R(A) V (or R(A)^T V) [+ beta * prev], beta read from beta_dev when non-null.
// skip (device int, may be null): when *skip != 0 the expand step writes nothing.
kpsb_status ra_apply(const float* psf, int s0, int s1, int n, int bc, const float* V, int ldv,
                     int nb, float* U, int ldu, int transpose, const float* prev, int ldp,
                     const double* beta_dev, float beta_host, const int* skip,
                     const RAScratch& scr, cudaStream_t st);
// The same in FP64 (PSF, vectors and scratch all double): the FP64 TSVD.
kpsb_status ra_apply(const double* psf, int s0, int s1, int n, int bc, const double* V, int ldv,
                     int nb, double* U, int ldu, int transpose, const double* prev, int ldp,
                     const double* beta_dev, double beta_host, const int* skip,
                     const RAScratch& scr, cudaStream_t st);

// ---- dense helpers (la.cu) --------------------------------------------------------------
// Scratch of a deterministic grid reduction (partials + counter).
struct RedScratch {
  double* part;           // >= RED_MAX_BLOCKS * width doubles
  unsigned int* counter;  // 1 (starts at zero)
};
static constexpr int RED_MAX_BLOCKS = 304;

// Templates on the basis element type T (float: SP TSVD; double: FP64 TSVD); instantiated
// in la.cu for both.
// h[i] = sum_r S[r + i ldS] v[r], i < m  (FP64 result; m <= 128).
template <typename T>
kpsb_status la_dot_block(const T* S, int ldS, int m, const T* v, long long N,
                         double* h, const RedScratch& red, const int* skip, cudaStream_t st);
// v -= S h (m columns); when norm_out != null also writes ||v||_2 (after the update).
template <typename T>
kpsb_status la_update(const T* S, int ldS, int m, const double* h, T* v, long long N,
                      double* norm_out, const RedScratch& red, const int* skip, cudaStream_t st);
// ||v||_2 into norm_out (FP64).
template <typename T>
kpsb_status la_norm(const T* v, long long N, double* norm_out, const RedScratch& red,
                    const int* skip, cudaStream_t st);
// v *= 1 / *norm (norm device FP64; zero norm leaves v unchanged).
template <typename T>
kpsb_status la_scale_inv(T* v, long long N, const double* norm, const int* skip, cudaStream_t st);
// G = Y^T Y (m x m FP64, column-major), Y N x m with leading dimension ldy; m <= 64.
template <typename T>
kpsb_status la_gram(const T* Y, int ldy, long long N, int m, double* G,
                    const RedScratch& red, cudaStream_t st);
// Out (N x kk, ldo) = Y (N x m, ldy) * T (m x kk FP64 column-major, ldt);  Out != Y.
template <typename TY, typename TO>
kpsb_status la_matmul_small(const TY* Y, int ldy, long long N, int m, const double* T,
                            int ldt, int kk, TO* Out, int ldo, cudaStream_t st);
// out[i] = in[i] converted.
template <typename TO, typename TI>
kpsb_status la_convert(const TI* in, TO* out, long long N, cudaStream_t st);
// One-sided Jacobi SVD of an m x nc FP64 matrix in device memory (one thread block):
// A = U diag(S) V^T, S descending.  m <= 128, nc <= 64, m >= nc.  sweeps may be null.
kpsb_status la_small_svd(const double* A, int lda, int m, int nc, double* U, double* S,
                         double* V, int* sweeps, cudaStream_t st);
// Standard normal values from Philox4x32-10 (counter = element index, key = seed) and the
// Box-Muller transform (computed in FP64, stored as T).
template <typename T>
kpsb_status la_randn(T* out, long long count, unsigned long long seed, cudaStream_t st);

// ---- EGKB parameters (kpbuild.cu, egkb_block.cu) ------------------------------------------
struct EgkbParams {
  int k_fixed;      // > 0: fixed rank
  int k_cap;
  int p;
  int k_min;
  double tau;       // relative tolerance (auto mode)
  double bd_tol;    // breakdown tolerance relative to bnorm
};

// ---- one-block EGKB for small images (egkb_block.cu) -----------------------------------
struct EbProblem {
  const double* psf;  // host, s0 x s1 column-major FP64
  int s0, s1, n, bc;
  EgkbParams P;
  int full_reorth;    // reorthogonalise the s_j too (the single-precision variant)
  int kpmax;          // k_cap + p
  const float* start_host;  // host start vector (n^2), or null: Philox from seed
  unsigned long long seed;
};
// Problems the one-block path takes: single precision, index-map R(A), n <= 128, the PSF
// staged in shared memory.
bool eb_eligible(int n, int s0, int s1);
// Builds every problem (all eligible) with one block per problem on stream st and waits for
// it.  outs[i] is null where problem i failed (st_out[i] / msg_out[i] say why).
kpsb_status egkb_block_build(const EbProblem* probs, int count, kpsb_kp_t* outs,
                             kpsb_status* st_out, std::string* msg_out, cudaStream_t st);
kpsb_status kp_handle_alloc(kpsb_kp_t* out, int n, int k, int kpsize);

// ---- KP operator handle ---------------------------------------------------------------
struct TCTables;  // tensor-core operand tables (kpgemm_tc.cu)

// ---- split Bregman state (sb.cu), shared with the serving loop -------------------------
struct SBScal;
struct SBProb {
  int n, iters, iso, fixed_inner, i_max;
  double mu, sqrt_mu, lam, thr, tau_cgls, tau_sb;
  double half_lam;        // lambda / 2
  const double* b;
  double *x, *xprev, *w, *f, *r1, *r2, *r3, *z1, *f1, *dx, *dy, *gx, *gy;
  double* q;              // tensor-core path: raw TV part of Ahat^T r (2 (Dx^T r2 + Dy^T r3) / lambda),
                          // kept in r2's storage instead of r2 and r3
  SBScal* sc;
  double* part;           // reduction partials
  unsigned int* counter;  // last-block counter
  float* xt;              // split planes of the next KP apply's input (tensor-core path):
                          // TF32 values in FP32 storage, or BF16 when xt_bf16
  float* z1f;             // FP32 KP-apply results (tensor-core path with split planes), else null
  float* f1f;
  float* wf;              // FP32 value of the CGLS direction w, the vector the forward apply
                          // sees (tensor-core path with split planes), else null
  int xt_bf16;            // the planes hold BF16 (BF16X3 / BF16X2 applies)
};
// Device-resident state of one problem; persists across sb_advance calls.
struct SBState {
  kpsb_kp* kp = nullptr;
  int n = 0, prec = 0, gemm_prec = 0;
  char* mem = nullptr;
  size_t bytes = 0;
  void* Z = nullptr;
  bool initialized = false;
  SBProb prob{};
};
size_t sb_state_bytes(int n, int k, int prec);
kpsb_status sb_state_init(SBState* S, kpsb_kp* kp, const double* b_dev, double* x_dev, double mu,
                          double lambda, double beta, int tv, int iters, const kpsb_sb_opts& o,
                          cudaStream_t st);
kpsb_status sb_advance(SBState* const* set, int count, int outer_steps, const kpsb_sb_opts& o,
                       cudaStream_t st);
kpsb_status sb_state_read(SBState* const* set, int count, std::vector<kpsb_sb_stats>& out,
                          std::vector<int>& done, cudaStream_t st);
void sb_state_free(SBState* S, cudaStream_t st);
kpsb_status sb_fill_defaults(const kpsb_sb_opts* opts, kpsb_sb_opts& o);

}  // namespace kpsb

struct kpsb_kp {
  int n = 0, k = 0, kp = 0;
  int device = 0;
  float* Ax = nullptr;     // k x n x n, column-major, unit Frobenius norm
  float* Ay = nullptr;     // k x n x n
  double* sigma_d = nullptr;  // k
  std::vector<double> sigma;  // host copy
  kpsb::TCTables* tc = nullptr;  // lazily built GEMM operand tables
  double* A_dense = nullptr;  // explicit operator A (kp_dense_blur): n^2 x n^2 FP64, k = 0
  std::mutex mu;
};

namespace kpsb {

// ---- KP apply (kpgemm.cu) ---------------------------------------------------------------
// One problem of a batched KP apply.
struct KPJob {
  const float* Ax;
  const float* Ay;
  const double* sigma;
  int n, k;
  const double* X;     // input n x n FP64
  double* Y;           // output n x n FP64
  void* Z;             // intermediate: k x n x n (FP64 or FP32 by precision)
  const int* active;   // skip when *active == 0 (may be null)
  // Tensor-core path only (zero for a plain apply):
  float* xt_ext;       // caller-maintained split planes of X ([2][n][n] row-major), or null
  float* yf;           // fused kernel: write the result in FP32 here instead of Y
  // Explicit operator (kp_dense_blur handles): A (n^2 x n^2 FP64); Z holds the partials
  const double* A;
};
// Y = sum sigma_i Ay_i X Ax_i^T (transpose 0) / sum sigma_i Ay_i^T X Ax_i (transpose 1)
// for every job (all with the same n).  jobs_d: device copy of the descriptors.
kpsb_status kp_apply_batch(const KPJob* jobs_d, int njobs, int n, int kmax, int transpose,
                           int prec, cudaStream_t st);
size_t kp_z_bytes(int n, int k, int prec);
// Explicit operator (dense.cu): Y = A X or A^T X for every job (all with the same n, J.A set,
// J.Z with dense_partials(n) doubles of scratch).
kpsb_status dense_apply_batch(const KPJob* jobs_d, int njobs, int n, int transpose, cudaStream_t st);
size_t dense_partials(int n);
// Work counters of the applies (sum of k n^3 and problem-applies over active problems),
// optionally reset; out may be null.
kpsb_status simt_work(unsigned long long* out, bool reset);
kpsb_status tc_work(unsigned long long* out, bool reset);

// Tensor-core path (kpgemm_tc.cu).  A plan holds the tensor maps and workspaces of one
// batch (forward and transpose jobs); applies reuse it.
struct TCPlan;
// Precisions that run on the tensor cores (TF32 and BF16 split modes).
inline bool prec_is_tc(int prec) {
  return prec == KPSB_P_TF32X3 || prec == KPSB_P_TF32X2 || prec == KPSB_P_BF16X3 || prec == KPSB_P_BF16X2;
}
inline bool prec_valid(int prec) { return prec >= KPSB_P_FP64 && prec <= KPSB_P_BF16X2; }
bool tc_supported(int n, int prec);
// Device bytes of a handle's tensor-core tables for one precision family, and of the
// per-problem workspace of a plan (split input planes and intermediate).
size_t tc_table_bytes(int n, int k, int prec);
size_t tc_plan_ws_bytes(int n, int k, int prec);
void tc_free(TCTables* t);
// shared_sms: the plan's applies run beside other parts of the same batch (the autotuner then
// ranks variants by SM time, not duration).
kpsb_status tc_plan_create(kpsb_kp** kps, const KPJob* fwd_h, const KPJob* bwd_h, int njobs, int n,
                           int prec, cudaStream_t st, TCPlan** out, bool shared_sms = false);
kpsb_status tc_plan_apply(TCPlan* P, int transpose, cudaStream_t st);
// True when the plan runs the fused kernel with CGLS epilogues (inputs split by the caller).
bool tc_plan_fused(const TCPlan* P);
// Kernel launches of one apply of the plan (split kernel when not supplied, then one fused
// launch or the two-stage pair).
int tc_plan_launches(const TCPlan* P);
void tc_plan_free(TCPlan* P, cudaStream_t st);
kpsb_status tc_check_error();
kpsb_status tc_apply_batch(kpsb_kp** kps, const KPJob* jobs_d, const KPJob* jobs_h, int njobs,
                           int n, int kmax, int transpose, int prec, cudaStream_t st);

}  // namespace kpsb

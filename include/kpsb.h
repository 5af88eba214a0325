/*
 * kpsb.h - C ABI of the GB300 (sm_103a) Kronecker-product-sum split Bregman library.
 *
 * Method: Alsubhi & Renaut, "Split Bregman isotropic and anisotropic image deblurring
 * with Kronecker product sum approximations using single precision enlarged-GKB or RSVD
 * algorithms to provide low rank truncated SVDs" (arXiv 2410.00233).  Section, algorithm
 * and equation numbers below refer to that paper.
 *
 * Conventions shared by every entry point
 *  - Images, PSFs, factors and blocks of vectors are COLUMN-MAJOR (the paper's vec/array,
 *    Sec. 1): element (i, j) of an m x n array is at [i + j*m].
 *  - Square images only (m1 = m2 = n1 = n2 = n, Sec. 5.1): R(A) is n^2 x n^2.
 *  - A PSF is s0 x s1 (rows x columns) with its centre tap at (s0/2, s1/2) (integer
 *    division).  Blur = convolution:  b(r,c) = sum_{a,b} P(a,b) x(ext(r-a+s0/2), ext(c-b+s1/2)).
 *    Zero boundary: out-of-range pixels are 0.  Reflexive boundary: half-sample mirror
 *    (x[-1] = x[0], x[n] = x[n-1]); requires s0/2 <= n, s1/2 <= n and s-1-s/2 <= n.
 *  - Every function returns a kpsb_status (0 = success, < 0 = error) and never throws;
 *    kpsb_last_error() gives a thread-local message for the last failure.
 *  - Host pointers ("host") are read/written synchronously: the call returns when the
 *    data is in place.  Device pointers ("dev") must be device-accessible memory of the
 *    current CUDA device; *_dev calls are asynchronous on the given stream (a
 *    cudaStream_t passed as void*, NULL = the legacy default stream) unless stated.
 *  - The caller owns every buffer it passes.  A kpsb_kp_t handle owns its device memory
 *    until kp_free().  Handles are not thread-safe: use one per thread or lock.
 *  - Plain pointers carry no sizes: every host or device buffer must hold at least the
 *    entries stated for it (the Python binding checks host arrays before the call).
 *
 * Environment switches (the first two only print; the third picks which kernel computes
 * the apply, where every variant gives the same bits and only the time changes; the fourth
 * picks the build path, whose two forms round differently):
 *   KPSB_TRACE=1        host phase trace of batched solves on stderr (plan ready, graph
 *                       instantiated and uploaded, launch, done; per stream)
 *   KPSB_TUNE_LOG=1     the tensor-core apply autotuner's timings on stderr
 *   KPSB_TC_VARIANT=v   pin the tensor-core apply variant (0 two-stage, 1 fused 64-column,
 *                       2 fused 32-column, 3 resident n = 128) instead of autotuning
 *   KPSB_EGKB_BLOCK=0   single-precision EGKB builds with n <= 128 use the multi-kernel path
 *                       instead of one thread block per problem (the default; both follow
 *                       Alg. 1 with the same arithmetic classes, summation orders differ)
 */
#ifndef KPSB_H
#define KPSB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KPSB_OK = 0,
  KPSB_EINVAL = -1,     /* invalid argument (size, pointer, option) */
  KPSB_ENOMEM = -2,     /* device or host allocation failed */
  KPSB_ECUDA = -3,      /* a CUDA runtime call or kernel launch failed */
  KPSB_ETIMEOUT = -4,   /* a bounded device wait ran out (see kpsb_last_error) */
  KPSB_EBREAKDOWN = -5, /* GKB/RSVD found no usable direction (k would be 0) */
  KPSB_ENOTCONV = -6,   /* iteration hit its limit where convergence was required */
  KPSB_EBUSY = -7,      /* admission refused: not enough free memory / slots */
  KPSB_ENOTFOUND = -8   /* unknown request id */
} kpsb_status;

/* Largest image side n accepted (n x n images; n^2 pixel indices fit 32 bits). */
#define KPSB_MAX_N 16384
enum { KPSB_BC_ZERO = 0, KPSB_BC_REFLEXIVE = 1 };
enum { KPSB_EGKB = 0, KPSB_RSVD = 1 };
enum { KPSB_ANISO = 0, KPSB_ISO = 1 };
/* Arithmetic of the Kronecker-sum GEMMs inside sb_solve / kp_apply (Sec. 4.2; the paper's
 * single precision, Sec. 4.4, carried to the tensor cores with split-precision recovery).
 * Vectors, stopping tests and shrinkage are FP64 in every mode.
 *  FP64  : FP64 FMA of the FP32 factors (exact in FP64) with FP64 images.
 *  FP32  : FP32 FMA, images rounded to FP32, FP32 accumulation.
 *  TF32X3: tensor cores (tcgen05 kind::tf32), each operand split into two TF32 parts,
 *          three products accumulated in FP32.
 *  TF32X2: tensor cores; the factors are used rounded once to TF32 (the same rounded
 *          operator in the forward and transpose applies, so the adjoint stays exact; the
 *          change of A_k is ~5e-4 relative, far below the KP truncation error) and the
 *          image is split into two TF32 parts: two products, half the factor traffic.
 *  BF16X3: tensor cores (tcgen05 kind::f16, BF16 operands, FP32 accumulation); each
 *          operand split into two BF16 parts (16 significant bits), three products
 *          (hi*hi + hi*lo + lo*hi): ~1e-5 relative per product, 1.5 TF32-product times
 *          of tensor work, 2-byte planes.
 *  BF16X2: tensor cores; the factors rounded once to BF16 (~4e-3 relative change of A_k,
 *          the same rounded operator in both directions), the image split into two BF16
 *          parts: two BF16 products, the smallest factor traffic.
 *  The tensor-core modes run for n >= 64 (image sides that are not a multiple of the
 *  128-row tile are masked); smaller sizes run the FP32 CUDA-core GEMM. */
enum { KPSB_P_FP64 = 0, KPSB_P_FP32 = 1, KPSB_P_TF32X3 = 2, KPSB_P_TF32X2 = 3, KPSB_P_BF16X3 = 4,
       KPSB_P_BF16X2 = 5 };
/* Shrinkage threshold of the d-subproblem argmin lambda^2||d-c||^2 + beta||d||_1
 * (Sec. 3.2-3.3): EXACT = beta/(2 lambda^2) (its exact minimiser), PAPER = beta/lambda^2
 * (the printed 1/gamma, which minimises with 2*beta). */
enum { KPSB_THR_EXACT = 0, KPSB_THR_PAPER = 1 };

typedef struct kpsb_kp* kpsb_kp_t;

/* Options of kp_build; zero-initialise and set what you need (0 selects the default). */
typedef struct {
  int p;             /* enlargement (EGKB) / oversampling (RSVD): k_p = k + p.  Default
                        max(2, ceil(k/4)) */
  int k_min;         /* automatic rank: smallest k the nu rule may pick (default 3) */
  int one_sided;     /* EGKB: 1 = reorthogonalise only the q_j (Alg. 1 step 6); default 0
                        = also the s_j (the single-precision variant, Sec. 4.4) */
  int power_iters;   /* RSVD power iterations q (Alg. 2 step 2), default 1 */
  unsigned long long seed; /* Philox4x32-10 seed for the start vector / test matrix */
  const float* start_host; /* optional host input: EGKB start vector y (n^2), or RSVD test
                        matrix F (n^2 x k_p, column-major).  NULL = Philox + Box-Muller */
  void* stream;      /* cudaStream_t for the work (NULL = legacy default stream) */
  int fp64;          /* 1: the TSVD in FP64 throughout (PSF, Krylov / sketch bases, R(A)
                        products; the paper's DP variant); 0 (default): single precision,
                        FP64 scalars.  The factors are stored in FP32 either way, sigma in FP64.
                        kp_build_dense supports single precision only. */
} kpsb_build_opts;

/* Options of sb_solve; zero-initialise, 0 selects the default. */
typedef struct {
  double beta;       /* TV weight beta; <= 0: beta = lambda^2/gamma with gamma = 2 (Sec. 5.3.1) */
  double tau_sb;     /* stop when RC_SB (5.2) < tau_sb; 0 (default) runs all `iters` steps */
  double tau_cgls;   /* CGLS stop on RC_CGLS (5.1) < tau_cgls; default 1e-4 */
  int i_max;         /* CGLS iteration limit I_max; default 100 */
  int fixed_inner;   /* 1: exactly i_max CGLS steps per outer step (no RC_CGLS test) */
  int prec;          /* KPSB_P_* for the KP GEMMs; default KPSB_P_FP64 */
  int threshold_rule;/* KPSB_THR_EXACT (default) or KPSB_THR_PAPER */
  void* stream;      /* cudaStream_t */
  int sub_batches;   /* sb_solve_batched: a size group of P problems is cut into this many
                        parts that run concurrently on their own streams, so one part's
                        FP64 vector kernels overlap another's tensor-core applies (results
                        do not change).  0 (default): min(4, P / 64), at least 1; 1: off. */
} kpsb_sb_opts;

typedef struct {
  int l_end;         /* outer (split Bregman) steps taken */
  int iota_total;    /* total CGLS steps */
  double rc_sb;      /* last RC_SB */
  int status;        /* kpsb_status of this solve */
} kpsb_sb_stats;

/* ---- Build: TSVD of R(A) and Terms(A_k) ------------------------------------------------
 * kp_build: approximate truncated SVD of the rearranged blur matrix R(A) (Sec. 2.1,
 * eq. (2.2)) in FP32 by EGKB (Alg. 1, Sec. 2.2) or RSVD (Alg. 2, Sec. 2.3), R(A) applied
 * matrix-free through the PSF's index map, then the KP terms (Theorem 2.1, Sec. 4.1.3):
 * A ~ sum_i sigma_i Ax_i (x) Ay_i, Ax_i = array(u_i, n, n), Ay_i = array(v_i, n, n).
 *   psf        host, s0 x s1 column-major FP64 (any scale; used as given)
 *   rank_or_tol >= 1: fixed rank k = (int)rank_or_tol.  In (0,1): EGKB only, automatic
 *              rank by the nu_j rule (eq. (2.6)) with relative tolerance tau = rank_or_tol
 *              (nu_i < tau*nu_3), capped at k <= 30.
 *   method     KPSB_EGKB or KPSB_RSVD.
 *   out        receives a new handle (device factors resident until kp_free).
 * The effective k may be smaller than asked when R(A) has smaller rank (R(A) = Kx P^T Ky^T,
 * so rank R(A) <= rank P <= min(s0, s1)):
 * the GKB recurrence stops at breakdown and RSVD drops null directions; kp_info reports
 * the k and k_p used.  Errors: EINVAL (n outside [2, KPSB_MAX_N], a PSF side outside
 * [1, 1024], a reflexive PSF overhang beyond the image, k < 1, k_p = k + p > 64, automatic
 * rank with RSVD; a zero-boundary PSF may be larger than the image),
 * ENOMEM, ECUDA, EBREAKDOWN (R(A) = 0).
 * Single-precision EGKB with n <= 128 and a PSF of at most 4096 entries (sides <= 128) runs
 * as one thread block per problem (the whole recurrence, the SVD of C and the Ritz vectors
 * in one launch pair), alone and in kp_build_batched alike, so a problem's factors do not
 * depend on its batch; other builds run as a sequence of grid-wide kernels. */
kpsb_status kp_build(const double* psf, int s0, int s1, int n, int bc, double rank_or_tol,
                     int method, const kpsb_build_opts* opts, kpsb_kp_t* out);

/* Size of a handle: n, number of terms k, enlarged size k_p; sigma (host, length >= k)
 * receives sigma_1 >= ... >= sigma_k (FP64).  Any output pointer may be NULL. */
kpsb_status kp_info(kpsb_kp_t kp, int* n, int* k, int* kp_size, double* sigma);

/* Host copies of the factors: Ax, Ay are k x (n x n) column-major FP32 (unit Frobenius
 * norm each; the first entry of largest magnitude of vec(Ay_i), in column-major order, is
 * positive), sigma FP64 (k).
 * Any pointer may be NULL. */
kpsb_status kp_get_factors(kpsb_kp_t kp, float* Ax, float* Ay, double* sigma);

/* Kronecker-product sum of a general operator (no PSF structure; the extension the paper
 * names as future work, Sec. 6): the TSVD of R(A) (Alg. 1 / Alg. 2, same options and
 * rank rules as kp_build) with R(A) read from the explicit matrix by eq. (2.2).  A: host,
 * N x N FP64 column-major (N = n^2, 2 <= n <= 128), copied once to the device in single
 * precision for the TSVD as in Sec. 1; block (i, j) of A (rows i n.., columns j n..) is row
 * i + j n of R(A), so the terms satisfy A ~= sum sigma_i Ax_i (x) Ay_i for column-major vec.
 * The caller keeps A; the handle owns the factors (kp_free). */
kpsb_status kp_build_dense(const double* A, int n, double rank_or_tol, int method,
                           const kpsb_build_opts* opts, kpsb_kp_t* out);

/* Handle of the exact blurring operator A itself as an explicit dense matrix (eq. (1.1);
 * the direct method of the paper's comparison, Sec. 4.3 case (i), Table 4 rows "A"):
 * A is n^2 x n^2 FP64 column-major on the device (2 GiB at n = 128), built from the PSF
 * (host, s0 x s1 column-major, centre (s0/2, s1/2)) with boundary bc exactly as kp_blur_dev
 * applies it.  kp_apply / kp_apply_dev (precision KPSB_P_FP64 only), sb_solve, sb_solve_dev
 * and sb_solve_batched accept the handle and run CGLS with A (always FP64, whatever the
 * precision option); kp_info reports k = 0; kp_get_factors fails with KPSB_EINVAL.
 * KPSB_EINVAL for n > 128 or a bad PSF / boundary, KPSB_ENOMEM if A does not fit.  Free
 * with kp_free. */
kpsb_status kp_dense_blur(const double* psf, int s0, int s1, int n, int bc, kpsb_kp_t* out);

/* Make a handle from given factors (host, same layout as kp_get_factors): lets a caller
 * run sb_solve on identical factors, or reuse cached ones. */
kpsb_status kp_from_factors(int n, int k, const float* Ax, const float* Ay,
                            const double* sigma, kpsb_kp_t* out);

/* KP apply (Sec. 4.2, eq. (4.3)): Y = sum_i sigma_i Ay_i X Ax_i^T (transpose = 0) or
 * X' = sum_i sigma_i Ay_i^T Y Ax_i (transpose = 1).  X, Y: n x n column-major FP64.
 * kp_apply: host pointers (synchronous).  kp_apply_dev: device pointers, async on
 * stream.  prec: KPSB_P_*.  X and Y must not overlap. */
kpsb_status kp_apply(kpsb_kp_t kp, const double* X, double* Y, int transpose, int prec);
kpsb_status kp_apply_dev(kpsb_kp_t kp, const double* X, double* Y, int transpose, int prec,
                         void* stream);

void kp_free(kpsb_kp_t kp);

/* ---- Split Bregman deblurring -----------------------------------------------------------
 * sb_solve: Alg. 3 (tv = KPSB_ANISO) or Alg. 4 (KPSB_ISO) with the KP operator of `kp`
 * in place of A:  min_x mu||A_k x - b||^2 + beta TV(x), splitting penalty lambda^2, L the
 * 1/2 forward difference with a zero last row (Sec. 5.3), x^(0) = b, d = g = 0.  Each
 * outer step solves (3.7) by CGLS (Alg. 5) from x = 0 on
 * Ahat = [sqrt(mu) A_k; lambda (L (x) I); lambda (I (x) L)], then shrinks (3.10)/(3.13)
 * and updates g (3.8)-(3.9).  iters = L_max.
 *   b, x_out: host n x n column-major FP64.  stats may be NULL.
 * Errors: EINVAL (mu <= 0, lambda <= 0, iters < 1), ENOMEM, ECUDA. */
kpsb_status sb_solve(kpsb_kp_t kp, const double* b, double mu, double lambda, int tv,
                     int iters, const kpsb_sb_opts* opts, double* x_out,
                     kpsb_sb_stats* stats);
/* Same with device b and x_out (n x n FP64 each), async on opts->stream; stats (host) is
 * filled when the call returns (the call synchronises the stream at its end). */
kpsb_status sb_solve_dev(kpsb_kp_t kp, const double* b, double mu, double lambda, int tv,
                         int iters, const kpsb_sb_opts* opts, double* x_out,
                         kpsb_sb_stats* stats);

/* ---- Batched (many independent problems in one set of launches) ------------------------ */
typedef struct {
  const double* psf; int s0, s1; int n; int bc; double rank_or_tol; int method;
  kpsb_build_opts opts;  /* opts.stream is ignored: the batch picks its streams */
} kpsb_problem;

/* Builds `count` handles: the problems of kp_build's one-block path share one launch pair
 * per chunk of 256 (one thread block each), the others run concurrently on internal streams.
 * outs[i] is NULL where problem i failed; the first error is returned.  The other problems
 * are still built, and their handles belong to the caller (kp_free each non-NULL outs[i],
 * also after an error).  Each handle equals the one kp_build gives for the same problem
 * alone. */
kpsb_status kp_build_batched(int count, const kpsb_problem* probs, kpsb_kp_t* outs);

typedef struct {
  kpsb_kp_t kp;       /* factors (n taken from it) */
  const double* b;    /* n x n FP64, host or device (see on_device) */
  double* x;          /* n x n FP64 output, host or device */
  double mu, lambda, beta; /* beta <= 0: lambda^2/2 */
  int tv;             /* KPSB_ANISO / KPSB_ISO */
  int iters;          /* L_max */
  kpsb_sb_stats* stats; /* may be NULL */
} kpsb_sb_job;

/* Solves `count` jobs together: jobs with the same n share every launch (grouped GEMMs
 * and vector kernels over problems, each problem with its own k and stopping state).
 * on_device = 1: b and x are device pointers.  opts gives the shared settings (tau,
 * i_max, prec, rule, stream).  The result of each job is bit-identical to its sb_solve
 * alone, in every precision: the kernels treat each problem on its own, reductions have a
 * fixed order, and every tensor-core apply variant issues the same MMAs per output element. */
kpsb_status sb_solve_batched(int count, const kpsb_sb_job* jobs, int on_device,
                             const kpsb_sb_opts* opts);

/* ---- Steps of the hot path, exposed for tests and composition -------------------------- */

/* Blur with the exact operator A (Sec. 1): B = A X (transpose = 0) or A^T X (1).
 * psf device FP64 s0 x s1; X, B device n x n FP64 (must not overlap).  Async. */
kpsb_status kp_blur_dev(const double* psf, int s0, int s1, int n, int bc, const double* X,
                        double* B, int transpose, void* stream);

/* Matrix-free block apply of R(A) (eq. (2.2), R(A) = Kx P^T Ky^T through the index map):
 * U = R(A) V (transpose = 0) or U = R(A)^T V (1).  psf device FP32 s0 x s1; V, U device
 * n^2 x nb FP32 with leading dimension ldv, ldu >= n^2 (must not overlap).  Its scratch
 * (per-tile partial sums, tap weights, counters) is allocated and freed on every call from the
 * stream-ordered pool (cudaMallocAsync / cudaFreeAsync on `stream`).  Async. */
kpsb_status kp_ra_apply_dev(const float* psf, int s0, int s1, int n, int bc, const float* V,
                            int ldv, int nb, float* U, int ldu, int transpose, void* stream);

/* kp_ra_apply_dev without any device allocation, for callers that cannot allocate during a
 * call: a real-time loop that must not pay for (or be synchronised by) cudaMalloc/cudaFree,
 * or a program that gives all device memory to its own pool up front.  The paper has no
 * counterpart; it is an integration convenience.  Arguments, layout and result are those of
 * kp_ra_apply_dev.  Scratch comes from one fixed 4 MiB array in device memory that every
 * device using the library keeps until the process exits; requests needing more
 * (n = 1024 with more than 15 vectors, n = 512 with more than 60) fail with KPSB_EINVAL
 * and a message.  Every call looks up the array's address on the current device; the first
 * call on a device also loads the library's device code there, so make that first call
 * before any stream capture.  `stream` must belong to the current device (KPSB_EINVAL
 * otherwise).  All calls share the array and it keeps the last call's contents (the call
 * clears what must start at zero), so calls that overlap on the GPU (different streams,
 * different host threads) race: serialise them. */
kpsb_status kp_ra_apply_noalloc_dev(const float* psf, int s0, int s1, int n, int bc,
                                    const float* V, int ldv, int nb, float* U, int ldu,
                                    int transpose, void* stream);

/* Materialise R(A) densely from the index map (n^2 x n^2 FP32, column-major, device;
 * n <= 128).  Each entry is a sum of PSF taps in a fixed order.  Async. */
kpsb_status kp_ra_materialize_dev(const float* psf, int s0, int s1, int n, int bc, float* R,
                                  void* stream);

/* Dense SVD of a small m x nc FP64 matrix on the device (one thread block, one-sided
 * Jacobi): A = U diag(S) V^T, S descending, m >= nc, m <= 128, nc <= 64.  Host pointers
 * (synchronous): A (m x nc), U (m x nc), S (nc), V (nc x nc), column-major.  sweeps
 * receives the Jacobi sweeps used (may be NULL). */
kpsb_status kpsb_small_svd(int m, int nc, const double* A, double* U, double* S, double* V,
                           int* sweeps);

/* ---- Serving: continuous batching of deblur requests (not in the paper) ----------------
 * A server keeps the split Bregman state of every admitted request resident on the device
 * and advances all of them together, round_steps outer steps per round; requests that
 * arrive while others run join at the next round, finished ones leave.  Admission is FIFO
 * while (a) fewer than max_active requests are resident and (b) their device memory
 * (state, and factors when the PSF is not cached) fits in budget_bytes; cached factors of
 * unused PSFs are evicted least-recently-used first when memory is needed.  Factors are
 * built (kp_build, start vector seeded by the PSF key) on a builder thread, so builds
 * overlap the running rounds, and cached by PSF key: a repeated PSF skips kp_build.  Each
 * result equals that of sb_solve on the same factors: per-problem kernels, fixed-order
 * reductions, and rounds that only regroup whole outer steps. */
typedef struct kpsb_server* kpsb_server_t;
typedef struct {
  const double* psf; int s0, s1;  /* host PSF, column-major, copied at submit */
  int n; int bc; double rank_or_tol; int method;
  const double* b;                /* host n x n FP64 data, copied at submit */
  double mu, lambda, beta;        /* beta <= 0: lambda^2 / 2 */
  int tv; int iters;              /* KPSB_ANISO / KPSB_ISO, outer steps L_max */
  int prec;                       /* KPSB_P_* of the KP GEMMs */
  unsigned long long psf_key;     /* cache key (and EGKB seed); 0: hash of the PSF and sizes */
} kpsb_request;
typedef struct {
  unsigned long long submitted, completed, failed, cache_hits, cache_misses, rounds;
  size_t bytes_in_use, peak_bytes;  /* device bytes accounted against the budget */
  int active, queued, cached;
} kpsb_srv_stats;
/* Starts the worker and builder threads on the current device. */
kpsb_status srv_create(size_t budget_bytes, int max_active, int round_steps, kpsb_server_t* out);
/* Queues a request (inputs copied); *id receives its id.  Requests that can never fit the
 * budget fail with KPSB_EBUSY (reported by srv_poll). */
kpsb_status srv_submit(kpsb_server_t s, const kpsb_request* req, unsigned long long* id);
/* Waits up to timeout_us (< 0: forever) for request id.  KPSB_OK: x_out (n x n host, may be
 * NULL), stats and latency_s (submit to result on the host, seconds) are filled and the
 * request is retired; KPSB_ETIMEOUT: still running; other codes: the request failed. */
kpsb_status srv_poll(kpsb_server_t s, unsigned long long id, long long timeout_us, double* x_out,
                     kpsb_sb_stats* stats, double* latency_s);
kpsb_status srv_stats(kpsb_server_t s, kpsb_srv_stats* out);
/* Stops the threads and frees everything, including requests never polled. */
void srv_destroy(kpsb_server_t s);

/* ---- Instrumentation ----------------------------------------------------------------- */
/* Kernels launched by this library in this process (all entry points, all threads). */
unsigned long long kpsb_kernel_launches(void);
/* enable = 1: clear the totals and record a CUDA event pair, on the launching stream,
 * around every Kronecker-sum GEMM apply (two kernel launches on the CUDA-core path, one
 * on the tensor-core path) and every split Bregman vector kernel, until called with
 * enable = 0.  While enabled, split Bregman runs its host-driven loop instead of one
 * CUDA graph (same kernels, same results). */
kpsb_status kpsb_gemm_timing(int enable);
/* Totals of the recorded applies (waits for their events): kernel launches, summed
 * device milliseconds, and algorithmic flops actually performed (4 k n^3 per problem per
 * apply, Sec. 4.2, counted on the device for problems still active, since the last
 * kpsb_gemm_timing(1)). */
kpsb_status kpsb_gemm_stats(unsigned long long* launches, double* ms, double* flops);
/* Device counters of the applies since the last kpsb_gemm_timing(1) (they run whether or
 * not timing is on): problem-applies performed and the sum of k n^3 over them. */
kpsb_status kpsb_apply_counts(unsigned long long* problem_applies, unsigned long long* kn3);
/* Totals of one timer category (same meaning as kpsb_gemm_stats; flops 0 for the vector
 * kernels): 0 KP applies, 1 CGLS ||z||^2 (Alg. 5 steps 3-4), 2 x and r updates with
 * RC_CGLS (steps 5-6), 3 f = Ahat^T r and tau (steps 7-9), 4 w = f + delta w (step 10),
 * 5 outer-step kernels (CGLS start, shrinkage of Alg. 3/4).  TSVD steps of kp_build /
 * kp_build_dense (Alg. 1 steps 3-6, Alg. 2): 6 R(A) products, 7 CGS2 reorthogonalisation
 * of the EGKB bases, 8 SVQB orthonormalisation of the RSVD blocks; for these three the
 * first value counts calls and the third holds ALGORITHMIC BYTES instead of flops (R(A):
 * the vectors read and written plus the PSF, or 4 n^4 per pass over an explicit A; CGS2:
 * 2 (2m + 3) N elements for m basis vectors; SVQB2: 10 m N elements); 9 the one-block EGKB
 * recurrence launches (n <= 128; one thread block per problem), whose third value is the sum of
 * the same R(A) and CGS2 byte counts over every problem of the launch.  KPSB_EINVAL for
 * another category. */
kpsb_status kpsb_timer_stats(int category, unsigned long long* launches, double* ms, double* flops);

/* Self-check of the exact integer binary32 <-> binary64 conversions that the split Bregman
 * vector kernels use in place of the conversion instructions (which GB300 issues to its FP64
 * pipe): every binary32 value widened, and n_random binary64 values (spread over the
 * binary32 subnormal, normal and overflow range, with round-to-nearest-even tie cases, zeros,
 * infinities and NaNs; drawn from `seed`) rounded, each compared bit for bit with the
 * hardware conversion on the current device (NaN against NaN).  *mismatches receives the
 * number that differ (0 expected).  Blocking; KPSB_ECUDA on a CUDA error. */
kpsb_status kpsb_conversion_check(unsigned long long n_random, unsigned long long seed,
                                  unsigned long long* mismatches);

/* The tensor-core apply variants the autotuner has chosen in this process (every variant
 * gives the same bits; the choice only moves time).  Writes up to max_rows rows of 7 ints
 * (n, precision, k_max, batch-size bucket (next power of two), caller-split planes 0/1,
 * shared SMs 0/1 (the batch ran as concurrent parts: variants ranked by SM time),
 * variant: 0 two-stage, 1 fused 64-column, 2 fused 32-column, 3 resident n = 128) to rows
 * (host, may be NULL) and returns the number of choices made. */
int kpsb_tuned_variants(int* rows, int max_rows);

/* Self-test of the bounded device waits behind KPSB_ETIMEOUT (the paper has no counterpart):
 * one thread waits on an mbarrier that nothing arrives at, through the same bounded-wait
 * routine as the tensor-core kernels, with a limit of about limit_us microseconds of SM clock
 * (1 .. 1000000) instead of their one second.  The wait runs out, the kernel records the
 * error flag as a timed-out GEMM pipeline does and returns, and the call returns KPSB_ETIMEOUT
 * with the pipeline's time-out message: that is the expected result, and the device stays
 * usable.  KPSB_OK would mean the wait completed; KPSB_EINVAL for a limit out of range.
 * Blocking; uses the current device. */
kpsb_status kpsb_wait_selftest(unsigned int limit_us);

/* Thread-local message for the last error of this thread ("" if none). */
const char* kpsb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KPSB_H */

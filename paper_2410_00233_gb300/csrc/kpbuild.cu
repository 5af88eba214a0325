// kp_build: TSVD of R(A) by EGKB (Alg. 1) or RSVD (Alg. 2) in FP32 on the device,
// FP64 bidiagonal / Gram SVDs on the device, then Terms(A_k) (Theorem 2.1, Sec. 4.1.3).
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <string>
#include <thread>

#include "kpsb_internal.cuh"

namespace kpsb {

static constexpr int KP_MAX = 64;   // largest enlarged size k_p
static constexpr int K_CAP = 30;    // automatic rank cap
static constexpr int NGATE = 2 * (KP_MAX + 4);

// Device-side scalar state of the GKB recurrence.
struct EgkbState {
  double alpha[KP_MAX + 4];  // alpha_j, j >= 1
  double t[KP_MAX + 4];      // t_j, j >= 1
  double zeta[KP_MAX + 4];
  double nu[KP_MAX + 4];
  double norm;     // last computed norm (t_j or alpha_j before acceptance)
  double coef_s;   // -alpha_{j-1}: coefficient of s_{j-1} in s_j
  double coef_q;   // -t_j: coefficient of q_{j-1} in q_j
  double bnorm;    // running lower bound of ||R(A)||
  int nq, ns;      // accepted q / s columns
  int k_sel, kp_target;
  int finished;    // 0 running, 1 complete, 2 breakdown in t, 3 breakdown in alpha
  int gate[NGATE]; // gate[ph] != 0: kernels of phase ph skip (ph = 2j: s-phase, 2j+1: q)
};

// Device address of a field of the device-resident state (no host dereference).
#define ST_FIELD(st, f) ((decltype(&((EgkbState*)0)->f))((char*)(st) + offsetof(EgkbState, f)))

// Decide after t_j (s-phase of step j).  j = 1 is the start vector.
__global__ void egkb_after_t(EgkbState* st, EgkbParams P, int j) {
  if (st->gate[2 * j]) return;
  double tj = st->norm;
  int stop = 0;
  if (j == 1) {
    st->t[1] = tj;
    st->ns = 1;
    if (!(tj > 0.0)) { st->finished = 2; st->norm = 0.0; stop = 1; }
  } else {
    st->bnorm = fmax(st->bnorm, tj);
    if (!(tj > P.bd_tol * st->bnorm)) {  // invariant subspace: s_j = 0, C's last row 0
      st->t[j] = 0.0;
      st->norm = 0.0;
      st->ns = j;
      st->finished = 2;
      stop = 1;
    } else {
      st->t[j] = tj;
      st->ns = j;
      if (st->kp_target > 0 && st->nq >= st->kp_target) { st->finished = 1; stop = 1; }
    }
  }
  st->coef_q = -st->t[j];
  if (stop)
    for (int ph = 2 * j + 1; ph < NGATE; ++ph) st->gate[ph] = 1;
}

// Decide after alpha_j (q-phase of step j): nu rule of Sec. 2.2 (eq. (2.6)).
__global__ void egkb_after_alpha(EgkbState* st, EgkbParams P, int j) {
  if (st->gate[2 * j + 1]) return;
  double aj = st->norm;
  st->bnorm = fmax(st->bnorm, aj);
  if (!(aj > P.bd_tol * st->bnorm) || (j == 1 && !(aj > 0.0))) {
    st->finished = 3;  // q_j is not accepted
    for (int ph = 2 * j + 2; ph < NGATE; ++ph) st->gate[ph] = 1;
    return;
  }
  st->alpha[j] = aj;
  st->nq = j;
  st->coef_s = -aj;
  if (j >= 2) {
    st->zeta[j] = aj * st->t[j];
    if (j >= 3) st->nu[j] = sqrt(st->zeta[j] * st->zeta[j - 1]);
  }
  if (P.k_fixed <= 0 && st->k_sel < 0 && j >= 4) {
    int i = j - 1;
    int kmin = P.k_min > 3 ? P.k_min : 3;
    if (i >= kmin && (st->nu[j] > st->nu[i] || st->nu[i] < P.tau * st->nu[3]))
      st->k_sel = i;
    else if (i >= P.k_cap)
      st->k_sel = P.k_cap;
    if (st->k_sel >= 0) {
      int kp = st->k_sel + P.p;
      st->kp_target = kp > st->nq ? kp : st->nq;
    }
  }
}

__global__ void egkb_init_state(EgkbState* st, EgkbParams P) {
  memset(st, 0, sizeof(EgkbState));
  st->k_sel = P.k_fixed > 0 ? P.k_fixed : -1;
  st->kp_target = P.k_fixed > 0 ? P.k_fixed + P.p : -1;
}

// Sign convention of Terms (Theorem 2.1 fixes each pair up to a common sign): the first
// entry of largest magnitude of vec(Ay_i) is made positive, flipping Ax_i with it.  Pass 1:
// every block finds its largest |Ay_i| entry (smallest index on ties) and merges it into one
// 64-bit key per term, (bits of |v|) << 32 | ~index, with atomicMax: the largest magnitude
// wins, then the smallest index.  Pass 2 flips the term where that entry is negative.
__global__ void sign_key_kernel(const float* __restrict__ Ay, long long N,
                                unsigned long long* __restrict__ keys) {
  const float* ay = Ay + (size_t)blockIdx.y * N;
  unsigned long long best = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
       e += (long long)gridDim.x * blockDim.x) {
    const unsigned long long key =
        ((unsigned long long)__float_as_uint(fabsf(ay[e])) << 32) | (0xFFFFFFFFull - (unsigned long long)e);
    best = key > best ? key : best;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
    best = other > best ? other : best;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(keys + blockIdx.y, best);
}

// Between the passes: the key of term i becomes its flip flag (read before any entry moves).
__global__ void sign_decide_kernel(const float* __restrict__ Ay, long long N, int k,
                                   unsigned long long* __restrict__ keys) {
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const long long idx = (long long)(0xFFFFFFFFull - (keys[i] & 0xFFFFFFFFull));
    keys[i] = Ay[(size_t)i * N + idx] < 0.f ? 1ull : 0ull;
  }
}

__global__ void sign_flip_kernel(float* __restrict__ Ax, float* __restrict__ Ay, long long N,
                                 const unsigned long long* __restrict__ flags) {
  if (!flags[blockIdx.y]) return;
  float* ay = Ay + (size_t)blockIdx.y * N;
  float* ax = Ax + (size_t)blockIdx.y * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N;
       e += (long long)gridDim.x * blockDim.x) {
    ay[e] = -ay[e];
    ax[e] = -ax[e];
  }
}

// keys: k zero-initialised 64-bit words of scratch (device).
static kpsb_status sign_fix(float* Ax, float* Ay, long long N, int k, unsigned long long* keys, cudaStream_t st) {
  KPSB_TRY_CUDA(cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * k, st));
  const int bx = (int)std::max(1LL, std::min<long long>((N + 255) / 256, 152));
  sign_key_kernel<<<dim3(bx, k), 256, 0, st>>>(Ay, N, keys);
  KPSB_CHECK_LAUNCH();
  sign_decide_kernel<<<1, 64, 0, st>>>(Ay, N, k, keys);
  KPSB_CHECK_LAUNCH();
  sign_flip_kernel<<<dim3(bx, k), 256, 0, st>>>(Ax, Ay, N, keys);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

// SVQB preparation: d_i = G_ii, Gs = D^{-1/2} G D^{-1/2} (zero rows where d_i = 0).
__global__ void svqb_scale_kernel(const double* G, int m, double* Gs, double* d) {
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e % m, j = e / m;
    double di = G[i + i * m], dj = G[j + j * m];
    Gs[e] = (di > 0.0 && dj > 0.0) ? G[e] / sqrt(di * dj) : 0.0;
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) d[i] = G[i + i * m];
}

// T = D^{-1/2} W Lambda^{-1/2}, dropping eigenvalues below tol * lambda_max (null
// directions of Y, i.e. the part of the space beyond the rank of R(A)).
__global__ void svqb_transform_kernel(const double* W, const double* lam, const double* d, int m,
                                      double tol, double* T) {
  double lmax = lam[0];
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e % m, j = e / m;
    double l = lam[j];
    double v = 0.0;
    if (l > tol * lmax && d[i] > 0.0) v = W[e] / sqrt(d[i]) / sqrt(l);
    T[e] = v;
  }
}

// RSVD final step: sigma_j = sqrt(lambda_j) of H H^T, T2 = U Sigma^{-1} (for V = H^T T2).
__global__ void rsvd_sigma_kernel(const double* lam, const double* U, int m, int k, double tol,
                                  double* sigma, double* T2) {
  double lmax = lam[0];
  for (int j = threadIdx.x; j < k; j += blockDim.x) sigma[j] = lam[j] > 0.0 ? sqrt(lam[j]) : 0.0;
  for (int e = threadIdx.x; e < m * k; e += blockDim.x) {
    int j = e / m;
    double l = lam[j];
    T2[e] = (l > tol * lmax) ? U[e] / sqrt(l) : 0.0;
  }
}

// ---- workspace ---------------------------------------------------------------------------------
// T: element type of the PSF and the Krylov / sketch bases (float: SP TSVD, double: FP64).
template <typename T>
struct BuildWork {
  char* base = nullptr;
  T* psf = nullptr;
  T* S = nullptr;    // N x (KP + 1)
  T* Q = nullptr;    // N x KP
  T* Tmp = nullptr;  // N x KP (RSVD temp)
  double* h = nullptr;  // 128
  double* small = nullptr;  // small matrices: C, U, S, V, G, ...
  EgkbState* st = nullptr;
  RAScratch ra;
  RedScratch red;
  const float* A32 = nullptr;  // general operator: explicit A in FP32 (no PSF), or null
};

// Algorithmic bytes of one R(A) product of nb vectors (element size el): the index-map form
// reads V, writes U (and reads prev when given) and reads the PSF; the explicit form streams
// A (4 n^4 bytes) once per group of up to 8 vectors.  Counted by the TSVD timers.
static double rop_bytes(bool dense, long long N, int nb, size_t el, bool prev, int s0, int s1) {
  const double vec = (double)el * N * nb * (prev ? 3.0 : 2.0);
  if (dense) return vec + 4.0 * (double)N * N * ((nb + 7) / 8);
  return vec + (double)el * s0 * s1;
}

// R(A) products of the build: the PSF's index map, or the explicit matrix when one is given
// (SP only).
static kpsb_status rop_apply(const BuildWork<float>& w, int s0, int s1, int n, int bc, const float* V, int ldv,
                             int nb, float* U, int ldu, int transpose, const float* prev, int ldp,
                             const double* beta_dev, float beta_host, const int* skip, cudaStream_t st) {
  const int slot = timer_begin(st);
  kpsb_status s =
      w.A32 ? ra_dense_apply(w.A32, n, V, ldv, nb, U, ldu, transpose, prev, ldp, beta_dev, beta_host, skip, st)
            : ra_apply(w.psf, s0, s1, n, bc, V, ldv, nb, U, ldu, transpose, prev, ldp, beta_dev, beta_host, skip,
                       w.ra, st);
  timer_end(slot, st, TIMER_RA, rop_bytes(w.A32 != nullptr, (long long)n * n, nb, sizeof(float), prev != nullptr,
                                          s0, s1), 1);
  return s;
}
static kpsb_status rop_apply(const BuildWork<double>& w, int s0, int s1, int n, int bc, const double* V,
                             int ldv, int nb, double* U, int ldu, int transpose, const double* prev, int ldp,
                             const double* beta_dev, double beta_host, const int* skip, cudaStream_t st) {
  const int slot = timer_begin(st);
  kpsb_status s = ra_apply(w.psf, s0, s1, n, bc, V, ldv, nb, U, ldu, transpose, prev, ldp, beta_dev, beta_host,
                           skip, w.ra, st);
  timer_end(slot, st, TIMER_RA, rop_bytes(false, (long long)n * n, nb, sizeof(double), prev != nullptr, s0, s1), 1);
  return s;
}

template <typename T> constexpr double eps_of();
template <> constexpr double eps_of<float>() { return 1.1920928955078125e-07; }
template <> constexpr double eps_of<double>() { return 2.220446049250313e-16; }

static size_t a256(size_t x) { return (x + 255) / 256 * 256; }

template <typename T>
static kpsb_status work_alloc(BuildWork<T>& w, int n, int s0, int s1, int kpmax, int nb_ra,
                              cudaStream_t st) {
  const size_t N = (size_t)n * n;
  const int smax = std::max(s0, s1);
  size_t off_psf = 0;
  size_t off_S = off_psf + a256(sizeof(T) * s0 * s1);
  size_t off_Q = off_S + a256(sizeof(T) * N * (kpmax + 1));
  size_t off_T = off_Q + a256(sizeof(T) * N * (kpmax + 1));
  size_t off_h = off_T + a256(sizeof(T) * N * (kpmax + 1));
  size_t off_small = off_h + a256(sizeof(double) * 256);
  size_t small_sz = a256(sizeof(double) * 12 * 130 * 66);
  size_t off_st = off_small + small_sz;
  size_t off_ra = off_st + a256(sizeof(EgkbState));
  size_t ra_bytes = ra_scratch_bytes(n, nb_ra, smax, sizeof(T));
  size_t off_red = off_ra + a256(ra_bytes);
  size_t red_bytes = a256(sizeof(double) * RED_MAX_BLOCKS * 64 * 64) + 256;
  size_t total = off_red + red_bytes;
  KPSB_TRY_CUDA(cudaMallocAsync((void**)&w.base, total, st));
  w.psf = (T*)(w.base + off_psf);
  w.S = (T*)(w.base + off_S);
  w.Q = (T*)(w.base + off_Q);
  w.Tmp = (T*)(w.base + off_T);
  w.h = (double*)(w.base + off_h);
  w.small = (double*)(w.base + off_small);
  w.st = (EgkbState*)(w.base + off_st);
  w.ra = ra_scratch_carve(w.base + off_ra, n, nb_ra, smax, sizeof(T));
  w.red.counter = (unsigned int*)(w.base + off_red);
  w.red.part = (double*)(w.base + off_red + 256);
  // counters must start at zero
  KPSB_TRY_CUDA(cudaMemsetAsync(w.ra.counters, 0, sizeof(unsigned int) * nb_ra, st));
  KPSB_TRY_CUDA(cudaMemsetAsync(w.red.counter, 0, sizeof(unsigned int), st));
  return KPSB_OK;
}

struct HostPsf {
  std::vector<float> f;
};

// CGS2: two passes of v -= B (B^T v) against m columns; the second pass also gives ||v||.
template <typename T>
static kpsb_status cgs2_run(const T* B, int ldb, int m, T* v, long long N, double* h,
                            double* norm_out, const RedScratch& red, const int* gate, cudaStream_t st) {
  if (m > 0) {
    KPSB_TRY(la_dot_block(B, ldb, m, v, N, h, red, gate, st));
    KPSB_TRY(la_update(B, ldb, m, h, v, N, nullptr, red, gate, st));
    KPSB_TRY(la_dot_block(B, ldb, m, v, N, h, red, gate, st));
    KPSB_TRY(la_update(B, ldb, m, h, v, N, norm_out, red, gate, st));
  } else {
    KPSB_TRY(la_norm(v, N, norm_out, red, gate, st));
  }
  return KPSB_OK;
}

template <typename T>
static kpsb_status cgs2(const T* B, int ldb, int m, T* v, long long N, double* h,
                        double* norm_out, const RedScratch& red, const int* gate, cudaStream_t st) {
  // algorithmic bytes: per pass the basis twice (dot, update) and v three times
  const int slot = timer_begin(st);
  const kpsb_status s = cgs2_run(B, ldb, m, v, N, h, norm_out, red, gate, st);
  timer_end(slot, st, TIMER_REORTH, m > 0 ? 2.0 * (2.0 * m + 3.0) * N * sizeof(T) : (double)N * sizeof(T), 1);
  return s;
}

// ---- EGKB ------------------------------------------------------------------------------------
// Steps (Alg. 1): t_1 = ||y||, s_1 = y/t_1; q_1 = R^T s_1 / alpha_1; for j >= 2:
//   s_j = R q_{j-1} - alpha_{j-1} s_{j-1} [reorthogonalised against s_1..s_{j-1}], t_j,
//   q_j = R^T s_j - t_j q_{j-1}, reorthogonalised against q_1..q_{j-1}, alpha_j, nu_j.
// Reorthogonalisation is classical Gram-Schmidt applied twice (CGS2), the blocked form
// of the modified Gram-Schmidt of the paper (same projection, at least as orthogonal).
// Copies a caller's FP32 start block (n^2 x m) into dst of the basis type.
template <typename T>
static kpsb_status upload_start(const float* host, T* dst, T* staging, long long count, cudaStream_t st) {
  if constexpr (sizeof(T) == sizeof(float)) {
    (void)staging;
    KPSB_TRY_CUDA(cudaMemcpyAsync(dst, host, sizeof(float) * count, cudaMemcpyHostToDevice, st));
    return KPSB_OK;
  } else {
    float* f = (float*)staging;  // staging holds count doubles, so count floats fit
    KPSB_TRY_CUDA(cudaMemcpyAsync(f, host, sizeof(float) * count, cudaMemcpyHostToDevice, st));
    return la_convert<double, float>(f, dst, count, st);
  }
}

template <typename T>
static kpsb_status egkb_run(BuildWork<T>& w, int n, int s0, int s1, int bc, const EgkbParams& P,
                            int full_reorth, int kpmax, const float* start_host,
                            unsigned long long seed, cudaStream_t st, int* nq_out, int* ns_out,
                            int* ksel_out, std::vector<double>& alpha, std::vector<double>& tvec) {
  const long long N = (long long)n * n;
  egkb_init_state<<<1, 1, 0, st>>>(w.st, P);
  KPSB_CHECK_LAUNCH();
  // s_1 = y / ||y||
  if (start_host) {
    KPSB_TRY(upload_start<T>(start_host, w.S, w.Tmp, N, st));
  } else {
    KPSB_TRY(la_randn<T>(w.S, N, seed, st));
  }
  int* gate = (int*)((char*)w.st + offsetof(EgkbState, gate));
  double* d_norm = ST_FIELD(w.st, norm);
  double* d_coef_s = ST_FIELD(w.st, coef_s);
  double* d_coef_q = ST_FIELD(w.st, coef_q);
  int* d_finished = ST_FIELD(w.st, finished);
  KPSB_TRY(la_norm(w.S, N, d_norm, w.red, gate + 2, st));
  egkb_after_t<<<1, 1, 0, st>>>(w.st, P, 1);
  KPSB_CHECK_LAUNCH();
  KPSB_TRY(la_scale_inv(w.S, N, d_norm, gate + 2, st));
  // q_1 = R^T s_1 / alpha_1
  KPSB_TRY(rop_apply(w, s0, s1, n, bc, w.S, (int)N, 1, w.Q, (int)N, 1, nullptr, 0, nullptr, (T)0,
                    gate + 3, st));
  KPSB_TRY(la_norm(w.Q, N, d_norm, w.red, gate + 3, st));
  egkb_after_alpha<<<1, 1, 0, st>>>(w.st, P, 1);
  KPSB_CHECK_LAUNCH();
  KPSB_TRY(la_scale_inv(w.Q, N, d_norm, gate + 3, st));

  int* h_fin = nullptr;
  KPSB_TRY_CUDA(cudaMallocHost((void**)&h_fin, sizeof(int)));
  *h_fin = 0;
  kpsb_status status = KPSB_OK;
  for (int j = 2; j <= kpmax + 1 && status == KPSB_OK; ++j) {
    T* sj = w.S + (size_t)(j - 1) * N;
    T* sjm1 = w.S + (size_t)(j - 2) * N;
    T* qjm1 = w.Q + (size_t)(j - 2) * N;
    T* qj = w.Q + (size_t)(j - 1) * N;
    const int* gs = gate + 2 * j;
    const int* gq = gate + 2 * j + 1;
    // s-phase
    status = rop_apply(w, s0, s1, n, bc, qjm1, (int)N, 1, sj, (int)N, 0, sjm1, (int)N,
                      d_coef_s, (T)0, gs, st);
    if (status) break;
    status = cgs2(w.S, (int)N, full_reorth ? j - 1 : 0, sj, N, w.h, d_norm, w.red, gs, st);
    if (status) break;
    egkb_after_t<<<1, 1, 0, st>>>(w.st, P, j);
    KPSB_CHECK_LAUNCH();
    status = la_scale_inv(sj, N, d_norm, gs, st);
    if (status) break;
    if (j == kpmax + 1) break;  // only s_{kp+1} is needed from the last step
    // q-phase
    status = rop_apply(w, s0, s1, n, bc, sj, (int)N, 1, qj, (int)N, 1, qjm1, (int)N,
                      d_coef_q, (T)0, gq, st);
    if (status) break;
    status = cgs2(w.Q, (int)N, j - 1, qj, N, w.h, d_norm, w.red, gq, st);
    if (status) break;
    egkb_after_alpha<<<1, 1, 0, st>>>(w.st, P, j);
    KPSB_CHECK_LAUNCH();
    status = la_scale_inv(qj, N, d_norm, gq, st);
    if (status) break;
    if (j % 4 == 0) {  // leave the loop early once the recurrence has finished
      cudaError_t e = cudaMemcpyAsync(h_fin, d_finished, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        set_error("egkb: %s", cudaGetErrorString(e));
        status = KPSB_ECUDA;
        break;
      }
      if (*h_fin) break;
    }
  }
  cudaFreeHost(h_fin);
  if (status) return status;
  EgkbState hs;
  KPSB_TRY_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(EgkbState), cudaMemcpyDeviceToHost, st));
  KPSB_TRY_CUDA(cudaStreamSynchronize(st));
  *nq_out = hs.nq;
  *ns_out = hs.ns;
  *ksel_out = hs.k_sel;
  alpha.assign(hs.alpha, hs.alpha + KP_MAX + 2);
  tvec.assign(hs.t, hs.t + KP_MAX + 2);
  return KPSB_OK;
}

kpsb_status kp_handle_alloc(kpsb_kp** out, int n, int k, int kpsize) {
  kpsb_kp* h = new (std::nothrow) kpsb_kp();
  if (!h) {
    set_error("out of host memory");
    return KPSB_ENOMEM;
  }
  h->n = n;
  h->k = k;
  h->kp = kpsize;
  cudaGetDevice(&h->device);
  size_t N = (size_t)n * n;
  cudaError_t e = cudaMalloc((void**)&h->Ax, sizeof(float) * N * k * 2 + sizeof(double) * k + 256);
  if (e != cudaSuccess) {
    delete h;
    set_error("handle allocation (%zu bytes): %s", sizeof(float) * N * k * 2, cudaGetErrorString(e));
    return KPSB_ENOMEM;
  }
  h->Ay = h->Ax + N * k;
  h->sigma_d = (double*)(((uintptr_t)(h->Ay + N * k) + 255) & ~(uintptr_t)255);
  *out = h;
  return KPSB_OK;
}

// Rank rule and breakdown tolerance of one EGKB build (k: the fixed rank, or the cap in the
// automatic mode tau > 0).
template <typename T>
static EgkbParams egkb_params(int k, double tau, const kpsb_build_opts& o) {
  EgkbParams P;
  P.k_fixed = tau > 0.0 ? 0 : k;
  P.k_cap = tau > 0.0 ? std::min(k, K_CAP) : k;
  P.p = o.p;
  P.k_min = o.k_min;
  P.tau = tau;
  P.bd_tol = 30.0 * eps_of<T>();
  return P;
}

template <typename T>
static kpsb_status build_egkb(const float* A32, const T* psf_host, int s0, int s1, int n, int bc, int k,
                              double tau, const kpsb_build_opts& o, cudaStream_t st, kpsb_kp** out) {
  const EgkbParams P = egkb_params<T>(k, tau, o);
  const int kpmax = P.k_cap + P.p;
  KPSB_REQUIRE(kpmax <= KP_MAX, "k + p = %d exceeds %d", kpmax, KP_MAX);
  const long long N = (long long)n * n;
  BuildWork<T> w;
  KPSB_TRY(work_alloc(w, n, s0, s1, kpmax, 1, st));
  w.A32 = A32;
  kpsb_status s = KPSB_OK;
  do {
    cudaError_t e = cudaMemcpyAsync(w.psf, psf_host, sizeof(T) * s0 * s1, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { set_error("psf upload: %s", cudaGetErrorString(e)); s = KPSB_ECUDA; break; }
    int nq = 0, ns = 0, ksel = 0;
    std::vector<double> alpha, tv;
    s = egkb_run(w, n, s0, s1, bc, P, !o.one_sided, kpmax, o.start_host, o.seed, st, &nq, &ns,
                 &ksel, alpha, tv);
    if (s) break;
    if (nq < 1) {
      set_error("EGKB: R(A) applied to the start vector vanishes");
      s = KPSB_EBREAKDOWN;
      break;
    }
    int kk = ksel > 0 ? std::min(ksel, nq) : std::min(P.k_cap, nq);
    // C ((nq+1) x nq lower bidiagonal) -> device, FP64 SVD (Alg. 1 step 15)
    const int m = nq + 1, nc = nq;
    std::vector<double> C((size_t)m * nc, 0.0);
    for (int i = 0; i < nc; ++i) {
      C[i + (size_t)i * m] = alpha[i + 1];
      C[i + 1 + (size_t)i * m] = tv[i + 2];
    }
    double* dC = w.small;
    double* dU = dC + 130 * 66;
    double* dSg = dU + 130 * 66;
    double* dV = dSg + 130;
    e = cudaMemcpyAsync(dC, C.data(), sizeof(double) * C.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { set_error("C upload: %s", cudaGetErrorString(e)); s = KPSB_ECUDA; break; }
    s = la_small_svd(dC, m, m, nc, dU, dSg, dV, nullptr, st);
    if (s) break;
    kpsb_kp* h = nullptr;
    s = kp_handle_alloc(&h, n, kk, nq);
    if (s) break;
    // Ritz vectors (steps 16-17): U = S_{nq+1} Uc[:, :k], V = Q_nq Vc[:, :k]
    s = la_matmul_small(w.S, (int)N, N, m, dU, m, kk, h->Ax, (int)N, st);
    if (!s) s = la_matmul_small(w.Q, (int)N, N, nc, dV, nc, kk, h->Ay, (int)N, st);
    if (!s) {
      s = sign_fix(h->Ax, h->Ay, N, kk, (unsigned long long*)w.h, st);
      e = s == KPSB_OK ? cudaGetLastError() : cudaSuccess;
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->sigma_d, dSg, sizeof(double) * kk, cudaMemcpyDeviceToDevice, st);
      h->sigma.resize(kk);
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->sigma.data(), dSg, sizeof(double) * kk, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { set_error("EGKB terms: %s", cudaGetErrorString(e)); s = KPSB_ECUDA; }
    }
    if (s) {
      kp_free(h);
      break;
    }
    *out = h;
  } while (0);
  cudaFreeAsync(w.base, st);
  return s;
}

// Orthonormalise the m columns of Y (N x m) in place by SVQB twice (Gram matrix, its
// eigen-decomposition, Y <- Y D^{-1/2} W Lambda^{-1/2}); null directions become zero.
template <typename T>
static kpsb_status svqb2_run(BuildWork<T>& w, T* Y, long long N, int m, cudaStream_t st);
// Timed wrapper; algorithmic bytes per pass: the Gram read, the transform's read and write,
// and the copy back (read and write) of the N x m block.
template <typename T>
static kpsb_status svqb2(BuildWork<T>& w, T* Y, long long N, int m, cudaStream_t st) {
  const int slot = timer_begin(st);
  const kpsb_status s = svqb2_run(w, Y, N, m, st);
  timer_end(slot, st, TIMER_QR, 2.0 * 5.0 * (double)m * N * sizeof(T), 1);
  return s;
}
template <typename T>
static kpsb_status svqb2_run(BuildWork<T>& w, T* Y, long long N, int m, cudaStream_t st) {
  double* G = w.small;
  double* Gs = G + 64 * 64;
  double* d = Gs + 64 * 64;
  double* U = d + 64;
  double* lam = U + 64 * 64;
  double* W = lam + 64;
  double* Tm = W + 64 * 64;
  for (int pass = 0; pass < 2; ++pass) {
    KPSB_TRY(la_gram(Y, (int)N, N, m, G, w.red, st));
    svqb_scale_kernel<<<1, 256, 0, st>>>(G, m, Gs, d);
    KPSB_CHECK_LAUNCH();
    KPSB_TRY(la_small_svd(Gs, m, m, m, U, lam, W, nullptr, st));
    svqb_transform_kernel<<<1, 256, 0, st>>>(W, lam, d, m, 1e-12, Tm);
    KPSB_CHECK_LAUNCH();
    KPSB_TRY(la_matmul_small(Y, (int)N, N, m, Tm, m, m, w.Tmp, (int)N, st));
    KPSB_TRY_CUDA(cudaMemcpyAsync(Y, w.Tmp, sizeof(T) * N * m, cudaMemcpyDeviceToDevice, st));
  }
  return KPSB_OK;
}

// ---- RSVD --------------------------------------------------------------------------------------
// Alg. 2 with q power iterations: Y = R F, orthonormalised after every apply of R or R^T
// (step 2-3), H^T = R^T Q (step 4), SVD of H through the eigen-decomposition of H H^T
// (k_p x k_p, FP64; step 5), U = Q U_H (step 6), V = H^T U_H Sigma^{-1}, truncation (step 7).
template <typename T>
static kpsb_status build_rsvd(const float* A32, const T* psf_host, int s0, int s1, int n, int bc, int k,
                              const kpsb_build_opts& o, cudaStream_t st, kpsb_kp** out) {
  const int kp = k + o.p;
  KPSB_REQUIRE(kp <= KP_MAX, "k + p = %d exceeds %d", kp, KP_MAX);
  const long long N = (long long)n * n;
  BuildWork<T> w;
  KPSB_TRY(work_alloc(w, n, s0, s1, kp, kp, st));
  w.A32 = A32;
  kpsb_status s = KPSB_OK;
  do {
    cudaError_t e = cudaMemcpyAsync(w.psf, psf_host, sizeof(T) * s0 * s1, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { set_error("psf upload: %s", cudaGetErrorString(e)); s = KPSB_ECUDA; break; }
    T* F = w.S;  // N x kp
    if (o.start_host) {
      s = upload_start<T>(o.start_host, F, w.Tmp, N * kp, st);
      if (s) break;
    } else {
      s = la_randn<T>(F, N * kp, o.seed, st);
      if (s) break;
    }
    T* Y = w.Q;
    s = rop_apply(w, s0, s1, n, bc, F, (int)N, kp, Y, (int)N, 0, nullptr, 0, nullptr, (T)0,
                 nullptr, st);
    if (!s) s = svqb2(w, Y, N, kp, st);
    for (int it = 0; it < o.power_iters && !s; ++it) {
      s = rop_apply(w, s0, s1, n, bc, Y, (int)N, kp, F, (int)N, 1, nullptr, 0, nullptr, (T)0,
                   nullptr, st);
      if (!s) s = svqb2(w, F, N, kp, st);
      if (!s) s = rop_apply(w, s0, s1, n, bc, F, (int)N, kp, Y, (int)N, 0, nullptr, 0, nullptr,
                           (T)0, nullptr, st);
      if (!s) s = svqb2(w, Y, N, kp, st);
    }
    if (s) break;
    // H^T = R^T Q  (N x kp) into F
    T* Ht = F;
    s = rop_apply(w, s0, s1, n, bc, Y, (int)N, kp, Ht, (int)N, 1, nullptr, 0, nullptr, (T)0,
                 nullptr, st);
    if (s) break;
    double* G = w.small;
    double* U = G + 64 * 64;
    double* lam = U + 64 * 64;
    double* W = lam + 64;
    double* sig = W + 64 * 64;
    double* T2 = sig + 64;
    s = la_gram(Ht, (int)N, N, kp, G, w.red, st);
    if (!s) s = la_small_svd(G, kp, kp, kp, U, lam, W, nullptr, st);
    if (s) break;
    rsvd_sigma_kernel<<<1, 256, 0, st>>>(lam, W, kp, k, 1e-12, sig, T2);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_error("rsvd: %s", cudaGetErrorString(e)); s = KPSB_ECUDA; break; }
    // effective k: drop directions with zero singular value (rank of R(A) < k)
    std::vector<double> hsig(k);
    e = cudaMemcpyAsync(hsig.data(), sig, sizeof(double) * k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { set_error("rsvd: %s", cudaGetErrorString(e)); s = KPSB_ECUDA; break; }
    int kk = 0;
    const double drop = sizeof(T) == sizeof(float) ? 1e-6 : 1e-13;  // below the arithmetic's resolution
    while (kk < k && hsig[kk] > drop * hsig[0]) ++kk;
    if (kk == 0) {
      set_error("RSVD: R(A) applied to the test matrix vanishes");
      s = KPSB_EBREAKDOWN;
      break;
    }
    kpsb_kp* h = nullptr;
    s = kp_handle_alloc(&h, n, kk, kp);
    if (s) break;
    s = la_matmul_small(Y, (int)N, N, kp, W, kp, kk, h->Ax, (int)N, st);  // U = Q U_H
    if (!s) s = la_matmul_small(Ht, (int)N, N, kp, T2, kp, kk, h->Ay, (int)N, st);
    if (!s) {
      s = sign_fix(h->Ax, h->Ay, N, kk, (unsigned long long*)w.h, st);
      e = s == KPSB_OK ? cudaGetLastError() : cudaSuccess;
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->sigma_d, sig, sizeof(double) * kk, cudaMemcpyDeviceToDevice, st);
      h->sigma.assign(hsig.begin(), hsig.begin() + kk);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { set_error("RSVD terms: %s", cudaGetErrorString(e)); s = KPSB_ECUDA; }
    }
    if (s) {
      kp_free(h);
      break;
    }
    *out = h;
  } while (0);
  cudaFreeAsync(w.base, st);
  return s;
}

}  // namespace kpsb

using namespace kpsb;

// Checks a build request and fills the option defaults (kp_build and kp_build_batched).
static kpsb_status build_args(const double* psf, int s0, int s1, int n, int bc, double rank_or_tol, int method,
                              const kpsb_build_opts* opts, kpsb_build_opts& o, int& k, double& tau) {
  KPSB_REQUIRE(psf, "null pointer");
  KPSB_TRY(ra_check(s0, s1, n, bc));
  KPSB_REQUIRE(method == KPSB_EGKB || method == KPSB_RSVD, "unknown method %d", method);
  KPSB_REQUIRE(rank_or_tol > 0.0 && isfinite(rank_or_tol), "rank_or_tol must be > 0");
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  tau = 0.0;
  if (rank_or_tol >= 1.0) {
    k = (int)rank_or_tol;
  } else {
    KPSB_REQUIRE(method == KPSB_EGKB, "automatic rank needs EGKB (RSVD takes a fixed k)");
    tau = rank_or_tol;
    k = K_CAP;
  }
  KPSB_REQUIRE(k >= 1 && k <= KP_MAX, "rank %d outside [1, %d]", k, KP_MAX);
  if (o.p <= 0) o.p = std::max(2, (k + 3) / 4);
  if (o.power_iters <= 0) o.power_iters = 1;
  if (o.k_min <= 0) o.k_min = 3;
  KPSB_REQUIRE(std::min(k, K_CAP) + o.p <= KP_MAX || tau == 0.0, "k_cap + p exceeds %d", KP_MAX);
  return KPSB_OK;
}

// Single-precision EGKB on small images runs as one thread block per problem (egkb_block.cu),
// alone and in batches alike; KPSB_EGKB_BLOCK=0 selects the multi-kernel path instead.
static bool use_block_path(int n, int s0, int s1, int method, const kpsb_build_opts& o) {
  if (method != KPSB_EGKB || o.fp64) return false;
  const char* f = getenv("KPSB_EGKB_BLOCK");
  if (f && f[0] == '0') return false;
  return eb_eligible(n, s0, s1);
}

static EbProblem eb_problem(const double* psf, int s0, int s1, int n, int bc, int k, double tau,
                            const kpsb_build_opts& o) {
  EbProblem e;
  e.psf = psf;
  e.s0 = s0;
  e.s1 = s1;
  e.n = n;
  e.bc = bc;
  e.P = egkb_params<float>(k, tau, o);
  e.full_reorth = !o.one_sided;
  e.kpmax = e.P.k_cap + e.P.p;
  e.start_host = o.start_host;
  e.seed = o.seed;
  return e;
}

// ---- C ABI ----------------------------------------------------------------------------------------
extern "C" kpsb_status kp_build(const double* psf, int s0, int s1, int n, int bc, double rank_or_tol,
                                int method, const kpsb_build_opts* opts, kpsb_kp_t* out) {
  clear_error();
  KPSB_REQUIRE(psf && out, "null pointer");
  *out = nullptr;
  kpsb_build_opts o;
  int k = 0;
  double tau = 0.0;
  KPSB_TRY(build_args(psf, s0, s1, n, bc, rank_or_tol, method, opts, o, k, tau));
  cudaStream_t st = (cudaStream_t)o.stream;
  if (use_block_path(n, s0, s1, method, o)) {
    const EbProblem ep = eb_problem(psf, s0, s1, n, bc, k, tau, o);
    kpsb_status ps = KPSB_OK;
    std::string msg;
    return egkb_block_build(&ep, 1, out, &ps, &msg, st);
  }
  if (o.fp64) {  // the TSVD in FP64 throughout (PSF, bases, R(A) products)
    std::vector<double> pd(psf, psf + (size_t)s0 * s1);
    if (method == KPSB_EGKB) return build_egkb<double>(nullptr, pd.data(), s0, s1, n, bc, k, tau, o, st, out);
    return build_rsvd<double>(nullptr, pd.data(), s0, s1, n, bc, k, o, st, out);
  }
  std::vector<float> pf((size_t)s0 * s1);
  for (size_t i = 0; i < pf.size(); ++i) pf[i] = (float)psf[i];
  if (method == KPSB_EGKB) return build_egkb<float>(nullptr, pf.data(), s0, s1, n, bc, k, tau, o, st, out);
  return build_rsvd<float>(nullptr, pf.data(), s0, s1, n, bc, k, o, st, out);
}

extern "C" kpsb_status kp_build_dense(const double* A, int n, double rank_or_tol, int method,
                                      const kpsb_build_opts* opts, kpsb_kp_t* out) {
  clear_error();
  KPSB_REQUIRE(A && out, "null pointer");
  *out = nullptr;
  KPSB_REQUIRE(n >= 2 && n <= 128, "explicit operator limited to n in [2, 128] (got %d)", n);
  KPSB_REQUIRE(method == KPSB_EGKB || method == KPSB_RSVD, "unknown method %d", method);
  KPSB_REQUIRE(rank_or_tol > 0.0 && isfinite(rank_or_tol), "rank_or_tol must be > 0");
  kpsb_build_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  double tau = 0.0;
  int k;
  if (rank_or_tol >= 1.0) {
    k = (int)rank_or_tol;
  } else {
    KPSB_REQUIRE(method == KPSB_EGKB, "automatic rank needs EGKB (RSVD takes a fixed k)");
    tau = rank_or_tol;
    k = K_CAP;
  }
  KPSB_REQUIRE(k >= 1 && k <= KP_MAX, "rank %d outside [1, %d]", k, KP_MAX);
  if (o.p <= 0) o.p = std::max(2, (k + 3) / 4);
  if (o.power_iters <= 0) o.power_iters = 1;
  if (o.k_min <= 0) o.k_min = 3;
  KPSB_REQUIRE(std::min(k, K_CAP) + o.p <= KP_MAX || tau == 0.0, "k_cap + p exceeds %d", KP_MAX);
  KPSB_REQUIRE(!o.fp64, "kp_build_dense runs the single-precision TSVD only");
  // the SP copy of A on the device (the R(A) products of the TSVD read it; Sec. 1)
  const size_t NN = (size_t)n * n * n * n;
  std::vector<float> a32(NN);
  for (size_t i = 0; i < NN; ++i) a32[i] = (float)A[i];
  float* dA = nullptr;
  KPSB_TRY_CUDA(cudaMalloc((void**)&dA, sizeof(float) * NN));
  cudaError_t e = cudaMemcpy(dA, a32.data(), sizeof(float) * NN, cudaMemcpyHostToDevice);
  kpsb_status s = KPSB_OK;
  if (e != cudaSuccess) {
    set_error("explicit operator upload: %s", cudaGetErrorString(e));
    s = KPSB_ECUDA;
  } else {
    const float one = 1.0f;  // unused 1 x 1 PSF: the products come from A
    cudaStream_t st = (cudaStream_t)o.stream;
    s = method == KPSB_EGKB ? build_egkb<float>(dA, &one, 1, 1, n, KPSB_BC_ZERO, k, tau, o, st, out)
                            : build_rsvd<float>(dA, &one, 1, 1, n, KPSB_BC_ZERO, k, o, st, out);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (s == KPSB_OK && e2 != cudaSuccess) {
      set_error("kp_build_dense: %s", cudaGetErrorString(e2));
      s = KPSB_ECUDA;
    }
  }
  cudaFree(dA);
  return s;
}

extern "C" kpsb_status kp_info(kpsb_kp_t kp, int* n, int* k, int* kp_size, double* sigma) {
  clear_error();
  KPSB_REQUIRE(kp, "null handle");
  if (n) *n = kp->n;
  if (k) *k = kp->k;
  if (kp_size) *kp_size = kp->kp;
  if (sigma) memcpy(sigma, kp->sigma.data(), sizeof(double) * kp->k);
  return KPSB_OK;
}

extern "C" kpsb_status kp_get_factors(kpsb_kp_t kp, float* Ax, float* Ay, double* sigma) {
  clear_error();
  KPSB_REQUIRE(kp, "null handle");
  KPSB_REQUIRE(!kp->A_dense, "an explicit-operator handle has no Kronecker factors");
  size_t bytes = sizeof(float) * (size_t)kp->n * kp->n * kp->k;
  if (Ax) KPSB_TRY_CUDA(cudaMemcpy(Ax, kp->Ax, bytes, cudaMemcpyDeviceToHost));
  if (Ay) KPSB_TRY_CUDA(cudaMemcpy(Ay, kp->Ay, bytes, cudaMemcpyDeviceToHost));
  if (sigma) memcpy(sigma, kp->sigma.data(), sizeof(double) * kp->k);
  return KPSB_OK;
}

extern "C" kpsb_status kp_from_factors(int n, int k, const float* Ax, const float* Ay,
                                       const double* sigma, kpsb_kp_t* out) {
  clear_error();
  KPSB_REQUIRE(Ax && Ay && sigma && out, "null pointer");
  KPSB_REQUIRE(n >= 2 && n <= KPSB_MAX_N && k >= 1 && k <= KP_MAX, "bad sizes n=%d k=%d", n, k);
  kpsb_kp* h = nullptr;
  KPSB_TRY(kp_handle_alloc(&h, n, k, k));
  size_t bytes = sizeof(float) * (size_t)n * n * k;
  cudaError_t e = cudaMemcpy(h->Ax, Ax, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->Ay, Ay, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->sigma_d, sigma, sizeof(double) * k, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    kp_free(h);
    set_error("kp_from_factors: %s", cudaGetErrorString(e));
    return KPSB_ECUDA;
  }
  h->sigma.assign(sigma, sigma + k);
  *out = h;
  return KPSB_OK;
}

extern "C" void kp_free(kpsb_kp_t kp) {
  if (!kp) return;
  if (kp->tc) tc_free(kp->tc);
  if (kp->Ax) cudaFree(kp->Ax);
  if (kp->A_dense) cudaFree(kp->A_dense);
  delete kp;
}

extern "C" kpsb_status kp_build_batched(int count, const kpsb_problem* probs, kpsb_kp_t* outs) {
  clear_error();
  KPSB_REQUIRE(count >= 0 && (count == 0 || (probs && outs)), "bad batch");
  if (count == 0) return KPSB_OK;
  int dev = 0;
  KPSB_TRY_CUDA(cudaGetDevice(&dev));
  std::vector<kpsb_status> st(count, KPSB_OK);
  std::vector<std::string> msg(count);
  // Problems of the one-block path share two launches per chunk; the others run through
  // kp_build on up to 8 host threads, each with its own stream, so their builds (and their few
  // host synchronisations) overlap on the device.
  std::vector<int> blk, rest;
  std::vector<EbProblem> ebp;
  for (int i = 0; i < count; ++i) {
    outs[i] = nullptr;
    kpsb_build_opts o;
    int k = 0;
    double tau = 0.0;
    const kpsb_problem& q = probs[i];
    st[i] = build_args(q.psf, q.s0, q.s1, q.n, q.bc, q.rank_or_tol, q.method, &q.opts, o, k, tau);
    if (st[i] != KPSB_OK) {
      msg[i] = kpsb_last_error();
      continue;
    }
    if (use_block_path(q.n, q.s0, q.s1, q.method, o)) {
      blk.push_back(i);
      ebp.push_back(eb_problem(q.psf, q.s0, q.s1, q.n, q.bc, k, tau, o));
    } else {
      rest.push_back(i);
    }
  }
  if (!blk.empty()) {
    cudaStream_t s = nullptr;
    KPSB_TRY_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    constexpr int CHUNK = 256;  // bounds the bases held at once (about 5 MB per problem at n = 128)
    for (size_t c0 = 0; c0 < blk.size(); c0 += CHUNK) {
      const int cnt = (int)std::min<size_t>(CHUNK, blk.size() - c0);
      std::vector<kpsb_kp_t> o2(cnt, nullptr);
      std::vector<kpsb_status> s2(cnt, KPSB_OK);
      std::vector<std::string> m2(cnt);
      const kpsb_status sc = egkb_block_build(ebp.data() + c0, cnt, o2.data(), s2.data(), m2.data(), s);
      const std::string chunk_msg = sc != KPSB_OK ? kpsb_last_error() : "";
      for (int u = 0; u < cnt; ++u) {
        const int i = blk[c0 + u];
        outs[i] = o2[u];
        st[i] = s2[u];
        if (s2[u] != KPSB_OK) msg[i] = m2[u].empty() ? chunk_msg : m2[u];
      }
    }
    cudaStreamDestroy(s);
  }
  const int NR = (int)rest.size();
  const int NT = std::min(NR, 8);
  auto worker = [&](int t) {
    cudaSetDevice(dev);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (int u = t; u < NR; u += NT) { st[rest[u]] = KPSB_ECUDA; msg[rest[u]] = "stream creation failed"; }
      return;
    }
    for (int u = t; u < NR; u += NT) {
      const int i = rest[u];
      kpsb_build_opts o = probs[i].opts;
      o.stream = s;
      st[i] = kp_build(probs[i].psf, probs[i].s0, probs[i].s1, probs[i].n, probs[i].bc,
                       probs[i].rank_or_tol, probs[i].method, &o, &outs[i]);
      if (st[i] != KPSB_OK) msg[i] = kpsb_last_error();
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> th;
  for (int t = 0; t < NT; ++t) th.emplace_back(worker, t);
  for (auto& x : th) x.join();
  for (int i = 0; i < count; ++i)
    if (st[i] != KPSB_OK) {
      set_error("problem %d: %s", i, msg[i].c_str());
      return st[i];
    }
  return KPSB_OK;
}

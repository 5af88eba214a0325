// Kronecker-sum GEMMs on the 5th-generation tensor cores (tcgen05, TMEM accumulators,
// TMA-fed shared memory, mbarrier pipeline), split-precision TF32 ("TF32x3"): every FP32
// operand a is split into a_hi = tf32(a) and a_lo = tf32(a - a_hi), and a*b is accumulated
// in FP32 as a_hi b_hi + a_hi b_lo + a_lo b_hi (error ~ FP32 rounding).
//
// One KP apply (Sec. 4.2, eq. (4.3)) per problem, forward Y = sum_i sigma_i Ay_i X Ax_i^T:
//   split : Xt = X^T as two TF32 planes (hi, lo), row-major.
//   stage1: for every term i,  D1[r][c] = sum_m Xt[r][m] T1_i[c][m]    (= Z_i(r, c))
//           T1_i[c][m] = sigma_i Ax_i(c, m)       (transpose apply: sigma_i Ax_i(m, c))
//           epilogue writes Zt[c][i n + r] as hi/lo planes.
//   stage2: D2[a][c] = sum_{i,r} T2[a][i n + r] Zt[c][i n + r]          (= Y(a, c))
//           T2[a][i n + r] = Ay_i(a, r)           (transpose apply: Ay_i(r, a))
//           epilogue writes Y column-major in FP64.
// Both stages are "C = A B^T" with both operands K-major (rows contiguous in K), which is
// the canonical tcgen05 operand form; the tables T1, T2 are built once per handle.
//
// BF16 modes (BF16X3, BF16X2) run the same two-stage kernel with BF16 planes (2 bytes, a
// 128-byte row holds 64 K values) and tcgen05.mma kind::f16 (K = 16 per instruction); the
// split is a_hi = bf16(a), a_lo = bf16(a - a_hi).  Image sides that are not a multiple of
// the tiles are handled by TMA's zero fill beyond the tensor extents (every leading
// dimension is padded to a multiple of 8 elements so the strides stay 16-byte multiples) and
// by masked epilogue stores.
//
// Kernel anatomy (128 threads, one 128 x BN output tile per CTA): warp 0 allocates BN TMEM
// columns; lane 0 of warp 0 issues TMA loads of 32-wide K slices (128-byte swizzle) into a
// ring of shared-memory stages; lane 0 of warp 1 issues tcgen05.mma (kind::tf32, M = 128,
// N = BN, K = 8) and releases each stage with tcgen05.commit; after the last MMA all four
// warps read their 32 TMEM lanes with tcgen05.ld and run the epilogue.  Every wait is
// bounded: on timeout the CTA records an error code, drains and frees TMEM, and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "kpsb_internal.cuh"

namespace kpsb {

// ------------------------------------------------------------------------------------------
// Tensor maps (driver entry point fetched through the runtime, no libcuda link needed)
// ------------------------------------------------------------------------------------------
typedef CUresult (*PFN_encodeTiled_t)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                       const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                       const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                       CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled_t encode_fn() {
  static PFN_encodeTiled_t fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_encodeTiled_t)p;
  });
  return fn;
}

// Row-major planes: dims (innermost first) {K, rows, planes[, terms]}, box {128 bytes of K,
// box_rows}: 32 FP32 (TF32) values or 64 BF16 values.
static kpsb_status make_map(CUtensorMap* m, const void* base, int rank, const cuuint64_t* dims,
                            const cuuint64_t* strides_bytes, int box_rows, bool bf16 = false) {
  PFN_encodeTiled_t enc = encode_fn();
  KPSB_REQUIRE(enc, "cuTensorMapEncodeTiled unavailable");
  cuuint32_t box[4] = {bf16 ? 64u : 32u, (cuuint32_t)box_rows, 1, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   (cuuint32_t)rank, (void*)base, dims,
                   strides_bytes, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d): rank %d dims %llu x %llu", (int)r, rank,
              (unsigned long long)dims[0], (unsigned long long)dims[1]);
    return KPSB_ECUDA;
  }
  return KPSB_OK;
}

// ------------------------------------------------------------------------------------------
// Device helpers: PTX wrappers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: gives up after limit_cycles of SM clock (false).
__device__ __forceinline__ bool mbar_wait_limit(uint64_t* bar, uint32_t parity, long long limit_cycles) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit_cycles) return false;
  }
  return true;
}
// The pipelines' waits: about a second of SM clock at most.
static constexpr long long TC_WAIT_CYCLES = 2000000000LL;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  return mbar_wait_limit(bar, parity, TC_WAIT_CYCLES);
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y, int z, int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B
// apart (SBO), version 1 (sm_100 family).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
  return d;
}

// Instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor: kind::f16 with BF16 A and B, D = F32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// D += A B with A read from tensor memory (M rows = TMEM lanes, K along columns) and B
// from shared memory.
__device__ __forceinline__ void mma_tf32_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc,
                                            uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accum));
}

// 32 consecutive columns of this thread's TMEM lane (no wait: call tmem_ld_wait before use).
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
      "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
      "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Two-part split of an FP32 value into the plane element type E: float planes hold TF32
// values (hi = tf32(v), lo = tf32(v - hi)); BF16 planes hold hi = bf16(v), lo = bf16(v - hi)
// (round to nearest even).
__device__ __forceinline__ void split2(float v, float& h, float& l) {
  h = tf32_round(v);
  l = tf32_round(v - h);
}
__device__ __forceinline__ void split2(float v, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  l = __float2bfloat16_rn(v - __bfloat162float(h));
}

// ------------------------------------------------------------------------------------------
// Jobs
// ------------------------------------------------------------------------------------------
struct alignas(128) TCJob {
  CUtensorMap m1A;   // Xt planes: {n, n, 2}
  CUtensorMap m1B;   // T1 planes: {n, n, 2, k} (box 128 rows, two-stage kernel)
  CUtensorMap m1F;   // T1 planes, box 64 rows (fused kernel, BN = 64)
  CUtensorMap m1G;   // T1 planes, box 32 rows (fused kernel, BN = 32)
  CUtensorMap m1R;   // T1 planes, box 128 rows (resident kernel, n = 128)
  CUtensorMap m2A;   // T2 planes: {k n, n, 2}
  CUtensorMap m2B;   // Zt planes: {k n, n, 2}
  const double* X;   // input image (n x n FP64, column-major)
  double* Y;         // output image
  void* Xt;          // [2][n][ldx] (float TF32 values or BF16)
  void* Zt;          // [2][n][ldz]
  int n, k, ldz, ldx;
  const int* active;
  float* Yf;         // when set (fused kernel): FP32 output instead of Y
  float* part;       // two-stage stage 2 split over K: FP32 partial tiles [split][tiles][BN][128]
  unsigned int* tctr;  // ... and one arrival counter per output tile (zero between launches)
};

// Leading dimensions of the planes: K extents padded to 8 elements, so every TMA stride is a
// multiple of 16 bytes for FP32 and BF16 planes alike.
static inline int pad8(long long x) { return (int)((x + 7) / 8 * 8); }
static inline bool prec_bf16(int prec) { return prec == KPSB_P_BF16X3 || prec == KPSB_P_BF16X2; }
// planes of the factor operand: 2 (split factors, three products) or 1 (rounded once)
static inline int prec_fpl(int prec) { return (prec == KPSB_P_TF32X3 || prec == KPSB_P_BF16X3) ? 2 : 1; }

// Tensor-core tables of one handle: [k][2][n][ld1] for stage 1, [2][n][ld2] for stage 2,
// forward and transpose; TF32 values in FP32 storage and, when a BF16 mode is used, BF16.
struct TCTables {
  float* T1f = nullptr;
  float* T1t = nullptr;
  float* T2f = nullptr;
  float* T2t = nullptr;
  __nv_bfloat16* B1f = nullptr;
  __nv_bfloat16* B1t = nullptr;
  __nv_bfloat16* B2f = nullptr;
  __nv_bfloat16* B2t = nullptr;
  int n = 0, k = 0, ld1 = 0, ld2 = 0;
};

void tc_free(TCTables* t) {
  if (!t) return;
  if (t->T1f) cudaFree(t->T1f);
  if (t->B1f) cudaFree(t->B1f);
  delete t;
}

// The two-stage kernel masks partial tiles, so any n >= 64 runs on the tensor cores; the
// fused and resident kernels need n a multiple of 128 (TF32 modes).
bool tc_supported(int n, int prec) { return prec_is_tc(prec) && n >= 64; }

size_t tc_table_bytes(int n, int k, int prec) {
  const size_t per = (size_t)2 * k * n * pad8(n) + (size_t)2 * n * pad8((long long)k * n);
  return per * 2 * (prec_bf16(prec) ? sizeof(__nv_bfloat16) : sizeof(float));
}

static size_t s2_split_bytes(int n, bool bf);  // stage-2 partial tiles and counters of one problem

size_t tc_plan_ws_bytes(int n, int k, int prec) {
  const size_t es = prec_bf16(prec) ? sizeof(__nv_bfloat16) : sizeof(float);
  return es * ((size_t)2 * n * pad8(n) + (size_t)2 * n * pad8((long long)k * n)) + s2_split_bytes(n, prec_bf16(prec)) +
         1024;
}

// ---- table build ---------------------------------------------------------------------------
template <typename E>
__global__ void tc_tables_kernel(const float* __restrict__ Ax, const float* __restrict__ Ay,
                                 const double* __restrict__ sigma, int n, int k, int ld1, int ld2, E* T1f,
                                 E* T1t, E* T2f, E* T2t) {
  const long long nn = (long long)n * n;
  const long long total = nn * k;
  const size_t pl1 = (size_t)n * ld1, pl2 = (size_t)n * ld2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / nn);
    long long rem = e % nn;
    int row = (int)(rem / n), col = (int)(rem % n);  // row-major position (row, col)
    const float* ax = Ax + (size_t)i * nn;
    const float* ay = Ay + (size_t)i * nn;
    float sg = (float)sigma[i];
    // stage 1 tables: T1_i[c][m]
    float f = sg * ax[row + (size_t)col * n];   // forward: sigma Ax_i(c = row, m = col)
    float t = sg * ax[col + (size_t)row * n];   // transpose: sigma Ax_i(m = col, c = row)
    size_t o1 = (size_t)i * 2 * pl1 + (size_t)row * ld1 + col;
    E h, l;
    split2(f, h, l);
    T1f[o1] = h;
    T1f[o1 + pl1] = l;
    split2(t, h, l);
    T1t[o1] = h;
    T1t[o1 + pl1] = l;
    // stage 2 tables: T2[a][i n + r], a = row, r = col
    float f2 = ay[row + (size_t)col * n];       // forward: Ay_i(a, r)
    float t2 = ay[col + (size_t)row * n];       // transpose: Ay_i(r, a)
    size_t o2 = (size_t)row * ld2 + (size_t)i * n + col;
    split2(f2, h, l);
    T2f[o2] = h;
    T2f[o2 + pl2] = l;
    split2(t2, h, l);
    T2t[o2] = h;
    T2t[o2 + pl2] = l;
  }
}

static kpsb_status tc_tables(kpsb_kp* kp, cudaStream_t st, bool bf, TCTables** out) {
  std::lock_guard<std::mutex> lk(kp->mu);
  if (!kp->tc) {
    TCTables* t = new TCTables();
    t->n = kp->n;
    t->k = kp->k;
    t->ld1 = pad8(kp->n);
    t->ld2 = pad8((long long)kp->k * kp->n);
    kp->tc = t;
  }
  TCTables* t = kp->tc;
  const int n = t->n, k = t->k;
  const size_t per1 = (size_t)2 * k * n * t->ld1, per2 = (size_t)2 * n * t->ld2;  // elements per table
  const long long total = (long long)k * n * n;
  const int nb = (int)std::min<long long>((total + 255) / 256, 152 * 8);
  cudaError_t e = cudaSuccess;
  if (!bf && !t->T1f) {
    float* b = nullptr;
    e = cudaMalloc((void**)&b, sizeof(float) * 2 * (per1 + per2));
    if (e != cudaSuccess) {
      set_error("tensor-core tables (%zu bytes): %s", sizeof(float) * 2 * (per1 + per2), cudaGetErrorString(e));
      return KPSB_ENOMEM;
    }
    tc_tables_kernel<float><<<nb, 256, 0, st>>>(kp->Ax, kp->Ay, kp->sigma_d, n, k, t->ld1, t->ld2, b, b + per1,
                                                b + 2 * per1, b + 2 * per1 + per2);
    count_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaFree(b);
      set_error("tensor-core tables: %s", cudaGetErrorString(e));
      return KPSB_ECUDA;
    }
    t->T1f = b;
    t->T1t = b + per1;
    t->T2f = b + 2 * per1;
    t->T2t = b + 2 * per1 + per2;
  }
  if (bf && !t->B1f) {
    __nv_bfloat16* b = nullptr;
    e = cudaMalloc((void**)&b, sizeof(__nv_bfloat16) * 2 * (per1 + per2));
    if (e != cudaSuccess) {
      set_error("BF16 tables (%zu bytes): %s", sizeof(__nv_bfloat16) * 2 * (per1 + per2), cudaGetErrorString(e));
      return KPSB_ENOMEM;
    }
    tc_tables_kernel<__nv_bfloat16><<<nb, 256, 0, st>>>(kp->Ax, kp->Ay, kp->sigma_d, n, k, t->ld1, t->ld2, b,
                                                        b + per1, b + 2 * per1, b + 2 * per1 + per2);
    count_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaFree(b);
      set_error("BF16 tables: %s", cudaGetErrorString(e));
      return KPSB_ECUDA;
    }
    t->B1f = b;
    t->B1t = b + per1;
    t->B2f = b + 2 * per1;
    t->B2t = b + 2 * per1 + per2;
  }
  *out = t;
  return KPSB_OK;
}

// ---- split + transpose of the input image -----------------------------------------------------
// Xt[r][m] = X(r, m) as hi/lo planes of E (row-major, leading dimension ldx), any n.
// grid = (32 x 32 tiles, problems).
template <typename E>
__global__ void tc_split_kernel(const TCJob* __restrict__ jobs) {
  const TCJob& J = jobs[blockIdx.y];
  if (J.active && !*J.active) return;
  const int n = J.n;
  const int tiles = (n + 31) / 32;
  const int tr = blockIdx.x % tiles, tm = blockIdx.x / tiles;
  if (tm >= tiles) return;
  __shared__ float t[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int j = ty; j < 32; j += 8) {
    int r = tr * 32 + tx, m = tm * 32 + j;
    t[j][tx] = (r < n && m < n) ? (float)J.X[r + (size_t)m * n] : 0.f;  // coalesced along r
  }
  __syncthreads();
  E* xt = (E*)J.Xt;
  const size_t plane = (size_t)n * J.ldx;
  for (int j = ty; j < 32; j += 8) {
    int r = tr * 32 + j, m = tm * 32 + tx;
    if (r < n && m < n) {
      E h, l;
      split2(t[tx][j], h, l);
      xt[(size_t)r * J.ldx + m] = h;  // coalesced along m
      xt[plane + (size_t)r * J.ldx + m] = l;
    }
  }
}

// ------------------------------------------------------------------------------------------
// The GEMM kernel
// ------------------------------------------------------------------------------------------
__device__ int g_tc_error = 0;  // set on a timed-out wait (read by the host after a solve)
// Work actually performed by the applies of this file: [0] sum of k n^3 over active
// problems, [1] active problem-applies (one increment per problem per apply).
__device__ unsigned long long g_tc_work[2] = {0, 0};

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing arrives at, with
// a short limit; the timed-out wait records the error flag exactly as a GEMM kernel does.
__global__ void tc_wait_selftest_kernel(long long limit_cycles, int* __restrict__ out) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const bool ok = mbar_wait_limit(&bar, 0, limit_cycles);
    if (!ok) atomicExch(&g_tc_error, 1);
    *out = ok ? 1 : 0;
  }
}

__device__ __forceinline__ void count_apply_work(int k, int n) {
  atomicAdd(&g_tc_work[0], (unsigned long long)k * n * n * n);
  atomicAdd(&g_tc_work[1], 1ull);
}

// FPL = planes of the factor operand (2: split factors, three products per K slice;
// 1: factors rounded once to TF32, two products).  The iterate operand always has two.
template <int BN, int STAGES, int STAGE, int FPL, bool BF = false>
struct TCCfg {
  static constexpr int KS = BF ? 64 : 32;     // K values in one 128-byte row
  static constexpr int A_BYTES = 128 * 128;  // 128 rows x 128 bytes
  static constexpr int B_BYTES = BN * 128;
  static constexpr int A_PLANES = STAGE == 1 ? 2 : FPL;  // stage 1: A = iterate, stage 2: A = factors
  static constexpr int B_PLANES = STAGE == 1 ? FPL : 2;
  static constexpr int STAGE_BYTES = A_PLANES * A_BYTES + B_PLANES * B_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr int TMEM_COLS = BN < 32 ? 32 : BN;
};

template <int BN, int STAGES, int STAGE, int FPL, bool BF>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const TCJob* __restrict__ jobs, int tiles_m) {
  using C = TCCfg<BN, STAGES, STAGE, FPL, BF>;
  using E = typename std::conditional<BF, __nv_bfloat16, float>::type;
  const TCJob& J = jobs[blockIdx.z];
  const int term = STAGE == 1 ? (int)blockIdx.y : 0;
  if (term >= J.k) return;
  if (J.active && !*J.active) return;
  if (STAGE == 2 && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) count_apply_work(J.k, J.n);
  const int n = J.n;
  const int m0 = (blockIdx.x % tiles_m) * 128;
  const int c0 = (blockIdx.x / tiles_m) * BN;
  if (m0 >= n || c0 >= n) return;
  const int KT = STAGE == 1 ? n : J.k * n;  // K extent (zero-filled past it)
  const int nkb_all = (KT + C::KS - 1) / C::KS;
  // stage 2 split over K (grid.y ranges, fixed by n): this CTA's K slices [kb0, kb1)
  const int S = STAGE == 2 ? (int)gridDim.y : 1, ks = STAGE == 2 ? (int)blockIdx.y : 0;
  const int kb0 = (int)((long long)nkb_all * ks / S), kb1 = (int)((long long)nkb_all * (ks + 1) / S);
  const bool has_k = kb1 > kb0;

  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    // the tensor maps live in global memory (written before the launch): acquire them for
    // the tensor-map proxy before the first copy
    const CUtensorMap* mA = STAGE == 1 ? &J.m1A : &J.m2A;
    const CUtensorMap* mB = STAGE == 1 ? &J.m1B : &J.m2B;
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)mA) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)mB) : "memory");
    for (int kb = kb0; kb < kb1; ++kb) {
      const int s = (kb - kb0) % STAGES, round = (kb - kb0) / STAGES;
      if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1)) {
        s_fail = 1;
        break;
      }
      unsigned char* st = smem + s * C::STAGE_BYTES;
      mbar_expect_tx(&full[s], C::STAGE_BYTES);
      const int kx = kb * C::KS;
      unsigned char* sb = st + C::A_PLANES * C::A_BYTES;
      if (STAGE == 1) {
        tma_load_3d(st, &J.m1A, &full[s], kx, m0, 0);
        tma_load_3d(st + C::A_BYTES, &J.m1A, &full[s], kx, m0, 1);
        for (int pl = 0; pl < C::B_PLANES; ++pl)
          tma_load_4d(sb + pl * C::B_BYTES, &J.m1B, &full[s], kx, c0, pl, term);
      } else {
        for (int pl = 0; pl < C::A_PLANES; ++pl)
          tma_load_3d(st + pl * C::A_BYTES, &J.m2A, &full[s], kx, m0, pl);
        tma_load_3d(sb, &J.m2B, &full[s], kx, c0, 0);
        tma_load_3d(sb + C::B_BYTES, &J.m2B, &full[s], kx, c0, 1);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    constexpr uint32_t idesc = BF ? idesc_bf16(128, BN) : idesc_tf32(128, BN);
    auto mma = [&](uint64_t a, uint64_t b, uint32_t acc) {
      if (BF) mma_bf16(tmem, a, b, idesc, acc);
      else mma_tf32(tmem, a, b, idesc, acc);
    };
    bool ok = true;
    for (int kb = kb0; kb < kb1; ++kb) {
      const int s = (kb - kb0) % STAGES, round = (kb - kb0) / STAGES;
      if (!mbar_wait(&full[s], round & 1)) {
        s_fail = 1;
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(smem + s * C::STAGE_BYTES);
      const uint32_t a_hi = sa, a_lo = sa + (C::A_PLANES == 2 ? C::A_BYTES : 0);
      const uint32_t b_hi = sa + C::A_PLANES * C::A_BYTES;
      const uint32_t b_lo = b_hi + (C::B_PLANES == 2 ? C::B_BYTES : 0);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {  // four 32-byte K steps (8 TF32 / 16 BF16) per row
        const uint32_t off = kk * 32;
        const uint32_t acc0 = (kb > kb0 || kk > 0) ? 1u : 0u;
        // Product order shared by every apply kernel: iterate lo x factor hi, iterate hi x
        // factor lo (split factors only), then hi x hi.  The iterate (X or Z, two planes) is
        // the A operand in stage 1 and the B operand in stage 2.
        const uint64_t a_h = sdesc_sw128(a_hi + off), b_h = sdesc_sw128(b_hi + off);
        if (STAGE == 1) {
          mma(sdesc_sw128(a_lo + off), b_h, acc0);
          if (FPL == 2) mma(a_h, sdesc_sw128(b_lo + off), 1u);
        } else {
          mma(a_h, sdesc_sw128(b_lo + off), acc0);
          if (FPL == 2) mma(sdesc_sw128(a_lo + off), b_h, 1u);
        }
        mma(a_h, b_h, 1u);
      }
      mma_commit(&empty[s]);  // stage s free once these MMAs have read it
    }
    if (ok) mma_commit(done);
  }
  __syncwarp();
  // ---- epilogue: all four warps ----
  bool ok = true;
  if (lane == 0) ok = mbar_wait(done, 0) && !s_fail;
  ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int row = m0 + warp * 32 + lane;  // TMEM lane = output row
    const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int cc = 0; cc < BN; cc += 16) {
      float v[16];
      tmem_ld16(tbase + cc, v);
      if (STAGE == 2 && S > 1) {
        // partial tile of this K range: [column][row], rows contiguous (coalesced)
        float* pt = J.part + ((size_t)ks * gridDim.x + blockIdx.x) * (size_t)(BN * 128);
#pragma unroll
        for (int j = 0; j < 16; ++j) pt[(size_t)(cc + j) * 128 + warp * 32 + lane] = has_k ? v[j] : 0.f;
      } else if (row < n) {
        if (STAGE == 1) {
          // D1[r][c] = Z_term(r, c) -> Zt[c][term n + r], hi/lo planes
          const size_t plane = (size_t)n * J.ldz;
          E* zt = (E*)J.Zt;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int c = c0 + cc + j;
            if (c < n) {
              E h, l;
              split2(v[j], h, l);
              size_t o = (size_t)c * J.ldz + (size_t)term * n + row;
              zt[o] = h;
              zt[plane + o] = l;
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int c = c0 + cc + j;
            if (c < n) {
              if (J.Yf) J.Yf[row + (size_t)c * n] = v[j];  // FP32 result for the CGLS kernels
              else J.Y[row + (size_t)c * n] = (double)v[j];
            }
          }
        }
      }
    }
  } else if (threadIdx.x == 0) {
    atomicExch(&g_tc_error, 1);
  }
  if (STAGE == 2 && S > 1) {
    // every CTA of the tile arrives (a failed one too, so the counter returns to zero; the
    // error flag then reports the launch); the last to arrive adds the partials in range order
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned prev = atomicAdd(&J.tctr[blockIdx.x], 1u);
      s_last = prev == (unsigned)S - 1;
      if (s_last) J.tctr[blockIdx.x] = 0u;  // no other CTA of this tile touches it again
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      // element i of the tile (column i / 128, row i % 128): 0 + p_0 + p_1 + ... in range order;
      // four elements per load, eight loads per partial in flight per thread
      constexpr int NF4 = BN * 128 / 4, U = 8;
      const float4* pb = (const float4*)(J.part + (size_t)blockIdx.x * (BN * 128));
      const size_t rs4 = (size_t)gridDim.x * (BN * 128 / 4);
#pragma unroll 1
      for (int base = threadIdx.x; base < NF4; base += 128 * U) {
        float4 a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) a[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int q = 0; q < S; ++q) {
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int i = base + u * 128;
            if (i < NF4) {
              const float4 t = __ldcg(pb + q * rs4 + i);
              a[u].x += t.x;
              a[u].y += t.y;
              a[u].z += t.z;
              a[u].w += t.w;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = base + u * 128;
          if (i >= NF4) continue;
          const int c = c0 + (4 * i) / 128, r = m0 + (4 * i) % 128;
          if (c >= n) continue;
          const float vv[4] = {a[u].x, a[u].y, a[u].z, a[u].w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            if (r + t >= n) break;
            if (J.Yf) J.Yf[r + t + (size_t)c * n] = vv[t];
            else J.Y[r + t + (size_t)c * n] = (double)vv[t];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (!ok && threadIdx.x == 0) {
    // drain: wait (bounded) for copies that may still be in flight into shared memory
    for (int s = 0; s < STAGES; ++s) mbar_wait(&full[s], 0);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::TMEM_COLS)
                 : "memory");
  }
}


// ------------------------------------------------------------------------------------------
// Fused apply: both stages in one CTA per (problem, BN-column tile); the intermediate
// Z_i(r, c) of a unit (term i, 128-row chunk rc of r) goes TMEM -> registers -> split TF32
// planes in shared memory (128-byte-swizzled K-major rows c, K = r) and is consumed there
// by the stage-2 MMAs, so it never reaches global memory.
//   units u = (i, rc), i < k, rc < R = n/128
//   S1(u): D1[u%2][r][c] = sum_m Xt[rc*128 + r][m] T1_i[c0 + c][m]       (K = n)
//   C(u) : Zs[c][r] = split(D1[u%2][r][c])                                (converter warps)
//   S2(u): D2[t][a][c] += sum_r T2[t*128 + a][i n + rc*128 + r] Zs[c][r]  (K = 128, every t)
// Issue order S1(0), S1(1), S2(0), S1(2), S2(1), ...: stage 1 of the next unit overlaps the
// conversion of the current one (two D1 buffers in TMEM).  Warps: 0 = TMA, 1 = MMA,
// 2..5 = converter and epilogue (TMEM lane quarters 2, 3, 0, 1).
// ------------------------------------------------------------------------------------------
static constexpr int FUSED_BN = 64;
static constexpr int FUSED_MAX_N = 384;  // largest n offered to the fused kernels (a multiple of 128)

template <int BN, int FPL>
struct FCfg {
  static constexpr int XA_BYTES = 128 * 128;         // one plane of a 128-row x 32-K slice
  static constexpr int TB_BYTES = BN * 128;          // one plane of a BN-row x 32-K slice
  static constexpr int S1_BYTES = 2 * XA_BYTES + FPL * TB_BYTES;  // Xt hi/lo + T1 planes
  static constexpr int S2_BYTES = FPL * XA_BYTES;                 // T2 planes
  static constexpr int SLOT = S1_BYTES > S2_BYTES ? S1_BYTES : S2_BYTES;
  static constexpr int ZS_PLANE = 4 * TB_BYTES;      // BN rows x 128 K: four 32-K sub-tiles
  static constexpr int ZS_BYTES = 2 * ZS_PLANE;      // hi, lo
  static constexpr int STAGES = 3;
  static constexpr int SMEM = STAGES * SLOT + ZS_BYTES + 1024 + 512;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that gives up at once when the CTA has already failed.
__device__ __forceinline__ bool fwait(uint64_t* bar, uint32_t parity, volatile int* fail) {
  if (*fail) return false;
  if (mbar_wait(bar, parity)) return true;
  *fail = 1;
  return false;
}

template <int BN, int FPL>
__global__ void __launch_bounds__(192, 1) tc_fused_kernel(const TCJob* __restrict__ jobs) {
  using C = FCfg<BN, FPL>;
  constexpr int STAGES = C::STAGES;
  const TCJob& J = jobs[blockIdx.y];
  if (J.active && !*J.active) return;
  const int n = J.n, k = J.k;
  const int c0 = blockIdx.x * BN;
  if (c0 >= n) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) count_apply_work(k, n);
  const int R = n / 128;
  const int U = k * R;
  const int nkb1 = n / 32;

  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* zs = smem + STAGES * C::SLOT;
  uint64_t* full = (uint64_t*)(zs + C::ZS_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* d1_full = empty + STAGES;
  uint64_t* d1_empty = d1_full + 2;
  uint64_t* zs_full = d1_empty + 2;
  uint64_t* zs_empty = zs_full + 1;
  uint64_t* d2_full = zs_empty + 1;
  uint32_t* tmem_slot = (uint32_t*)(d2_full + 1);
  __shared__ int s_fail_v;
  volatile int* s_fail = &s_fail_v;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)((R + 2) * BN)) ncols <<= 1;
  if (threadIdx.x == 0) {
    s_fail_v = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&d1_full[b], 1);
      mbar_init(&d1_empty[b], 4);
    }
    mbar_init(zs_full, 4);
    mbar_init(zs_empty, 1);
    mbar_init(d2_full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = idesc_tf32(128, BN);

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: slots in the MMA's consumption order ----
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)&J.m1A) : "memory");
    const CUtensorMap* mF = BN == 64 ? &J.m1F : &J.m1G;  // T1 slices with BN-row boxes
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)mF) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)&J.m2A) : "memory");
    int si = 0;
    bool ok = true;
    for (int v = 0; v <= U && ok; ++v) {
      if (v < U) {
        const int i = v / R, rc = v % R;
        for (int kb = 0; kb < nkb1 && ok; ++kb, ++si) {
          const int s = si % STAGES, round = si / STAGES;
          if (round > 0 && !fwait(&empty[s], (round - 1) & 1, s_fail)) { ok = false; break; }
          unsigned char* st = smem + s * C::SLOT;
          mbar_expect_tx(&full[s], C::S1_BYTES);
          tma_load_3d(st, &J.m1A, &full[s], kb * 32, rc * 128, 0);
          tma_load_3d(st + C::XA_BYTES, &J.m1A, &full[s], kb * 32, rc * 128, 1);
          for (int pl = 0; pl < FPL; ++pl)
            tma_load_4d(st + 2 * C::XA_BYTES + pl * C::TB_BYTES, mF, &full[s], kb * 32, c0, pl, i);
        }
      }
      if (v >= 1 && ok) {
        const int u = v - 1, i = u / R, rc = u % R;
        for (int t = 0; t < R && ok; ++t)
          for (int q = 0; q < 4 && ok; ++q, ++si) {
            const int s = si % STAGES, round = si / STAGES;
            if (round > 0 && !fwait(&empty[s], (round - 1) & 1, s_fail)) { ok = false; break; }
            unsigned char* st = smem + s * C::SLOT;
            mbar_expect_tx(&full[s], C::S2_BYTES);
            for (int pl = 0; pl < FPL; ++pl)
              tma_load_3d(st + pl * C::XA_BYTES, &J.m2A, &full[s], i * n + rc * 128 + q * 32, t * 128, pl);
          }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    int si = 0;
    bool ok = true;
    for (int v = 0; v <= U && ok; ++v) {
      if (v < U) {
        const uint32_t d1 = tmem + (uint32_t)((R + (v & 1)) * BN);
        if (v >= 2 && !fwait(&d1_empty[v & 1], ((v >> 1) - 1) & 1, s_fail)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int kb = 0; kb < nkb1; ++kb, ++si) {
          const int s = si % STAGES, round = si / STAGES;
          if (!fwait(&full[s], round & 1, s_fail)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(smem + s * C::SLOT);
          const uint32_t a_hi = sa, a_lo = sa + C::XA_BYTES;
          const uint32_t b_hi = sa + 2 * C::XA_BYTES, b_lo = b_hi + (FPL == 2 ? C::TB_BYTES : 0);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t off = kk * 32, acc0 = (kb > 0 || kk > 0) ? 1u : 0u;
            mma_tf32(d1, sdesc_sw128(a_lo + off), sdesc_sw128(b_hi + off), idesc, acc0);
            if (FPL == 2) mma_tf32(d1, sdesc_sw128(a_hi + off), sdesc_sw128(b_lo + off), idesc, 1u);
            mma_tf32(d1, sdesc_sw128(a_hi + off), sdesc_sw128(b_hi + off), idesc, 1u);
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&d1_full[v & 1]);
      }
      if (v >= 1) {
        const int u = v - 1;
        if (!fwait(zs_full, u & 1, s_fail)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t z_hi = smem_u32(zs), z_lo = z_hi + C::ZS_PLANE;
        for (int t = 0; t < R && ok; ++t) {
          const uint32_t d2 = tmem + (uint32_t)(t * BN);
          for (int q = 0; q < 4; ++q, ++si) {
            const int s = si % STAGES, round = si / STAGES;
            if (!fwait(&full[s], round & 1, s_fail)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa = smem_u32(smem + s * C::SLOT);
            const uint32_t a_hi = sa, a_lo = sa + (FPL == 2 ? C::XA_BYTES : 0);
            const uint32_t zq = q * C::TB_BYTES;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint32_t off = kk * 32;
              const uint32_t acc0 = (u > 0 || q > 0 || kk > 0) ? 1u : 0u;
              mma_tf32(d2, sdesc_sw128(a_hi + off), sdesc_sw128(z_lo + zq + off), idesc, acc0);
              if (FPL == 2) mma_tf32(d2, sdesc_sw128(a_lo + off), sdesc_sw128(z_hi + zq + off), idesc, 1u);
              mma_tf32(d2, sdesc_sw128(a_hi + off), sdesc_sw128(z_hi + zq + off), idesc, 1u);
            }
            mma_commit(&empty[s]);
          }
        }
        if (!ok) break;
        mma_commit(zs_empty);
      }
    }
    if (ok) mma_commit(d2_full);
  } else if (warp >= 2) {
    // ---- converter, then epilogue ----
    const int quarter = warp & 3;
    const int rl = quarter * 32 + lane;  // TMEM lane = row of the 128-row chunk
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    bool ok = true;
    for (int u = 0; u < U && ok; ++u) {
      if (!fwait(&d1_full[u & 1], (u >> 1) & 1, s_fail)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float v[BN];
#pragma unroll
      for (int c = 0; c < BN; c += 16) tmem_ld16(tmem + lane_base + (uint32_t)((R + (u & 1)) * BN + c), v + c);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&d1_empty[u & 1]);
      if (u >= 1 && !fwait(zs_empty, (u - 1) & 1, s_fail)) { ok = false; break; }
      // Zs[c][r]: sub-tile q = r / 32, 128-byte row c, 16-byte chunk ((r % 32) / 4) ^ (c % 8)
      unsigned char* zrow = zs + (rl >> 5) * C::TB_BYTES;
      const int ch = (rl & 31) >> 2, w4 = (rl & 3) * 4;
#pragma unroll
      for (int c = 0; c < BN; ++c) {
        const float h = tf32_round(v[c]);
        const int off = c * 128 + ((ch ^ (c & 7)) << 4) + w4;
        *(float*)(zrow + off) = h;
        *(float*)(zrow + C::ZS_PLANE + off) = tf32_round(v[c] - h);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(zs_full);
    }
    if (ok && fwait(d2_full, 0, s_fail)) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int t = 0; t < R; ++t) {
        float v[BN];
#pragma unroll
        for (int c = 0; c < BN; c += 16) tmem_ld16(tmem + lane_base + (uint32_t)(t * BN + c), v + c);
        const int a = t * 128 + rl;
        if (J.Yf) {  // FP32 result (the accumulation is FP32): no FP64 work in this kernel
#pragma unroll
          for (int c = 0; c < BN; ++c) J.Yf[a + (size_t)(c0 + c) * n] = v[c];
        } else {
#pragma unroll
          for (int c = 0; c < BN; ++c) J.Y[a + (size_t)(c0 + c) * n] = (double)v[c];
        }
      }
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*s_fail && threadIdx.x == 0) {
    atomicExch(&g_tc_error, 1);
    for (int s = 0; s < STAGES; ++s) mbar_wait(&full[s], 0);  // bounded drain of copies in flight
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// ------------------------------------------------------------------------------------------
// Resident apply for n = 128: a persistent grid (one CTA per SM) takes problems from a
// global counter (the TMA thread claims the next one and hands its index to the MMA and
// converter warps through a 4-slot ring in shared memory; -1 ends the walk; the last CTA
// to finish resets the counter for the next launch).  Per problem the iterate is kept in shared memory
// and the intermediate in tensor memory.  Both stages are computed transposed so that the
// intermediate can be the A operand of stage 2 straight from TMEM:
//   S1(i): D1[c][r]  = sum_m T1_i[c][m] Xt[r][m]         (= Z_i(r, c); A = T1_i, B = Xt)
//   C(i) : Zh/Zl[c][r] = split(D1[c][r])                   (TMEM -> registers -> TMEM)
//   S2(i): D2[c][a] += sum_r Z[c][r] T2[a][i n + r]       (A = Z in TMEM, B = T2)
// and Y(a, c) = D2[c][a]: TMEM lane c holds column c of Y, which the epilogue stores as 128
// contiguous floats.  TMEM columns: D1 [0, 128), Zh [128, 256), Zl [256, 384), D2 [384, 512).
// Shared memory: Xt hi/lo (128 KB) and a ring of 32-wide K slices of T1 / T2 (16 KB per
// plane) in the order the MMAs consume them: S1(0), S1(1), S2(0), S1(2), S2(1), ...
// Overlap: the converter releases D1 as soon as it has read it (S1(i + 1) runs while Z(i)
// is written); the next problem's iterate loads once the last stage-1 MMAs of the current
// one have completed, and its first MMAs run while the converter stores the current result.
// Warps: 0 = TMA, 1 = MMA, 2..5 = converter and epilogue (TMEM lane quarters 2, 3, 0, 1).
// Barrier phases follow a CTA-wide term counter g and problem counter j.
// ------------------------------------------------------------------------------------------
template <int FPL>
struct RCfg {
  static constexpr int TILE = 128 * 128;                 // 128 rows x 32 K x 4 bytes
  static constexpr int X_BYTES = 2 * 4 * TILE;           // hi, lo planes; 4 K slices each
  static constexpr int SLOT = FPL * TILE;
#ifndef KPSB_RES_RING_KB
#define KPSB_RES_RING_KB 96
#endif
  // ring of 16 KB planes: 96 KB gives 6 (FPL 1) or 3 (FPL 2) slots
  static constexpr int STAGES = KPSB_RES_RING_KB * 1024 / SLOT;
  static constexpr int SMEM = X_BYTES + STAGES * SLOT + 1024 + 512;
};

template <int FPL>
__global__ void __launch_bounds__(192, 1) tc_resident_kernel(const TCJob* __restrict__ jobs, int njobs,
                                                             int* __restrict__ queue) {
  using C = RCfg<FPL>;
  constexpr int STAGES = C::STAGES;
  constexpr int n = 128;

  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* xs = smem;                       // Xt planes
  unsigned char* ring = smem + C::X_BYTES;
  uint64_t* full = (uint64_t*)(ring + STAGES * C::SLOT);
  uint64_t* empty = full + STAGES;
  uint64_t* x_full = empty + STAGES;  // [4]: K slice kb of the iterate (hi and lo planes) loaded
  uint64_t* x_free = x_full + 4;
  uint64_t* d1_full = x_free + 1;
  uint64_t* d1_free = d1_full + 1;
  uint64_t* z_full = d1_free + 1;
  uint64_t* z_free = z_full + 1;
  uint64_t* d2_full = z_free + 1;
  uint64_t* d2_free = d2_full + 1;
  uint64_t* pq = d2_free + 1;  // [4]: problem index published
  uint32_t* tmem_slot = (uint32_t*)(pq + 4);
  __shared__ int s_fail_v;
  __shared__ int s_idx[4];
  volatile int* s_fail = &s_fail_v;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s_fail_v = 0;
    for (int q = 0; q < STAGES; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    for (int q = 0; q < 4; ++q) mbar_init(&pq[q], 1);
    for (int q = 0; q < 4; ++q) mbar_init(&x_full[q], 1);
    mbar_init(x_free, 1);
    mbar_init(d1_full, 1);
    mbar_init(d1_free, 4);
    mbar_init(z_full, 4);
    mbar_init(z_free, 1);
    mbar_init(d2_full, 1);
    mbar_init(d2_free, 4);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t t_d1 = tmem, t_zh = tmem + 128, t_zl = tmem + 256, t_d2 = tmem + 384;
  constexpr uint32_t idesc = idesc_tf32(128, 128);
  // a problem is processed when its CGLS is active and it has the size this kernel tiles
  auto live = [&](const TCJob& J) { return J.n == n && !(J.active && !*J.active); };
  // consumers: index of the j-th problem of this CTA (-1: none left); false on a failed wait
  auto next_problem = [&](int j, int* p) -> bool {
    if (!fwait(&pq[j & 3], (j >> 2) & 1, s_fail)) return false;
    *p = *(volatile int*)&s_idx[j & 3];
    return true;
  };

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    int si = 0, j = 0;
    bool ok = true;
    for (;; ++j) {
      int p;
      do {
        p = atomicAdd(queue, 1);
      } while (p < njobs && !live(jobs[p]));
      if (p >= njobs || !ok) p = -1;
      s_idx[j & 3] = p;
      mbar_arrive(&pq[j & 3]);  // release: the index is visible to whoever waits on pq
      if (p < 0) break;
      const TCJob& J = jobs[p];
      const int k = J.k;
      count_apply_work(k, n);
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)&J.m1A) : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)&J.m1R) : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"((uint64_t)&J.m2A) : "memory");
      // the iterate buffer is free once the previous problem's stage-1 MMAs have completed
      if (j > 0 && !fwait(x_free, (j - 1) & 1, s_fail)) { ok = false; break; }
      // slots in consumption order: S1(0), then S1(i + 1), S2(i) for every i; each K slice
      // of the iterate is requested just before the S1(0) table slice it meets, so the first
      // MMAs start once 32 KB of the iterate has landed
      for (int v = -1; v < k && ok; ++v) {
        const int i1 = v + 1;
        for (int part = 0; part < 2 && ok; ++part) {
          const bool s1 = part == 0;
          if (s1 && i1 >= k) continue;
          if (!s1 && v < 0) continue;
          for (int kb = 0; kb < 4; ++kb, ++si) {
            if (v < 0) {
              mbar_expect_tx(&x_full[kb], 2 * C::TILE);
              for (int pl = 0; pl < 2; ++pl)
                tma_load_3d(xs + (pl * 4 + kb) * C::TILE, &J.m1A, &x_full[kb], kb * 32, 0, pl);
            }
            const int q = si % STAGES, round = si / STAGES;
            if (round > 0 && !fwait(&empty[q], (round - 1) & 1, s_fail)) { ok = false; break; }
            unsigned char* st = ring + q * C::SLOT;
            mbar_expect_tx(&full[q], C::SLOT);
            for (int pl = 0; pl < FPL; ++pl) {
              if (s1) tma_load_4d(st + pl * C::TILE, &J.m1R, &full[q], kb * 32, 0, pl, i1);
              else    tma_load_3d(st + pl * C::TILE, &J.m2A, &full[q], v * n + kb * 32, 0, pl);
            }
          }
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    int si = 0, g = 0, j = 0;  // ring slot, CTA-wide term, problem
    bool ok = true;
    const uint32_t x_hi = smem_u32(xs), x_lo = x_hi + 4 * C::TILE;
    // S1 of CTA-wide term gi: D1 = T1 Xt^T, products T1hi*Xlo, T1lo*Xhi, T1hi*Xhi; xw: the
    // problem's first term, which also waits for each K slice of the iterate
    auto stage1 = [&](int gi, bool xw) -> bool {
      if (gi >= 1) {
        if (!fwait(d1_free, (gi - 1) & 1, s_fail)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      for (int kb = 0; kb < 4; ++kb, ++si) {
        const int q = si % STAGES, round = si / STAGES;
        if (!fwait(&full[q], round & 1, s_fail)) return false;
        if (xw && !fwait(&x_full[kb], j & 1, s_fail)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t t_hi = smem_u32(ring + q * C::SLOT), t_lo = t_hi + (FPL == 2 ? C::TILE : 0);
        const uint32_t xh = x_hi + kb * C::TILE, xl = x_lo + kb * C::TILE;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          // same product order as the other kernels: X lo x T hi, X hi x T lo, hi x hi
          const uint32_t off = kk * 32, acc0 = (kb > 0 || kk > 0) ? 1u : 0u;
          mma_tf32(t_d1, sdesc_sw128(t_hi + off), sdesc_sw128(xl + off), idesc, acc0);
          if (FPL == 2) mma_tf32(t_d1, sdesc_sw128(t_lo + off), sdesc_sw128(xh + off), idesc, 1u);
          mma_tf32(t_d1, sdesc_sw128(t_hi + off), sdesc_sw128(xh + off), idesc, 1u);
        }
        mma_commit(&empty[q]);
      }
      mma_commit(d1_full);
      return true;
    };
    // S2 of term gi (problem term i): D2 += Z T2^T, products Zlo*T2hi, Zhi*T2lo, Zhi*T2hi
    auto stage2 = [&](int gi, int i) -> bool {
      if (!fwait(z_full, gi & 1, s_fail)) return false;
      if (i == 0 && j > 0 && !fwait(d2_free, (j - 1) & 1, s_fail)) return false;  // D2 read out
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int kb = 0; kb < 4; ++kb, ++si) {
        const int q = si % STAGES, round = si / STAGES;
        if (!fwait(&full[q], round & 1, s_fail)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t b_hi = smem_u32(ring + q * C::SLOT), b_lo = b_hi + (FPL == 2 ? C::TILE : 0);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t off = kk * 32, col = (uint32_t)(kb * 32 + kk * 8);
          const uint32_t acc0 = (i > 0 || kb > 0 || kk > 0) ? 1u : 0u;
          mma_tf32_ta(t_d2, t_zl + col, sdesc_sw128(b_hi + off), idesc, acc0);
          if (FPL == 2) mma_tf32_ta(t_d2, t_zh + col, sdesc_sw128(b_lo + off), idesc, 1u);
          mma_tf32_ta(t_d2, t_zh + col, sdesc_sw128(b_hi + off), idesc, 1u);
        }
        mma_commit(&empty[q]);
      }
      mma_commit(z_free);
      return true;
    };
    for (; ok; ++j) {
      int p;
      if (!next_problem(j, &p)) { ok = false; break; }
      if (p < 0) break;
      const TCJob& J = jobs[p];
      const int k = J.k;
      ok = stage1(g, true);
      if (ok && k == 1) mma_commit(x_free);
      for (int i = 0; i < k && ok; ++i) {
        if (i + 1 < k) {
          ok = stage1(g + i + 1, false);
          if (ok && i + 2 == k) mma_commit(x_free);  // last stage-1 MMAs of this problem issued
        }
        if (ok) ok = stage2(g + i, i);
      }
      if (ok) mma_commit(d2_full);
      g += k;
    }
  } else if (warp >= 2) {
    // ---- converter, then epilogue ----
    const int quarter = warp & 3;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    const int c = quarter * 32 + lane;  // TMEM lane: column of Y
    int g = 0;
    bool ok = true;
    for (int j = 0; ok; ++j) {
      int p;
      if (!next_problem(j, &p)) { ok = false; break; }
      if (p < 0) break;
      const TCJob& J = jobs[p];
      const int k = J.k;
      uint32_t v[128];
      for (int i = 0; i < k && ok; ++i, ++g) {
        if (!fwait(d1_full, g & 1, s_fail)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 4; ++q) tmem_ld32_nowait(t_d1 + lane_base + q * 32, v + 32 * q);
        tmem_ld_wait();
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(d1_free);  // S1 of the next term may overwrite D1
        if (g >= 1) {
          if (!fwait(z_free, (g - 1) & 1, s_fail)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          uint32_t h[32];  // hi plane, then (after its store has issued) the lo plane
#pragma unroll
          for (int t = 0; t < 32; ++t) h[t] = __float_as_uint(tf32_round(__uint_as_float(v[32 * q + t])));
          tmem_st32(t_zh + lane_base + q * 32, h);
#pragma unroll
          for (int t = 0; t < 32; ++t)
            h[t] = __float_as_uint(tf32_round(__uint_as_float(v[32 * q + t]) - __uint_as_float(h[t])));
          tmem_st32(t_zl + lane_base + q * 32, h);
        }
        tmem_st_wait();
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(z_full);
      }
      if (!ok || !fwait(d2_full, j & 1, s_fail)) { ok = false; break; }
      // epilogue: column c of Y from TMEM lane c; D2 is free for the next problem once read
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int q = 0; q < 4; ++q) tmem_ld32_nowait(t_d2 + lane_base + q * 32, v + 32 * q);
      tmem_ld_wait();
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(d2_free);
      if (J.Yf) {
        float4* y = (float4*)(J.Yf + (size_t)c * n);
#pragma unroll
        for (int q = 0; q < 32; ++q)
          y[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                             __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
      } else if (((uintptr_t)J.Y & 15) == 0) {  // caller's FP64 output: vector stores when aligned
        double2* y = (double2*)(J.Y + (size_t)c * n);
#pragma unroll
        for (int q = 0; q < 64; ++q)
          y[q] = make_double2((double)__uint_as_float(v[2 * q]), (double)__uint_as_float(v[2 * q + 1]));
      } else {
        double* y = J.Y + (size_t)c * n;
#pragma unroll
        for (int q = 0; q < 128; ++q) y[q] = (double)__uint_as_float(v[q]);
      }
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*s_fail && threadIdx.x == 0) {
    atomicExch(&g_tc_error, 1);
    for (int q = 0; q < 4; ++q) mbar_wait(&x_full[q], 0);  // bounded drain of copies in flight
    for (int q = 0; q < STAGES; ++q) mbar_wait(&full[q], 0);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
  if (threadIdx.x == 0) {  // the last CTA out resets the problem counter for the next launch
    __threadfence();
    if (atomicAdd(queue + 1, 1) == (int)gridDim.x - 1) {
      atomicExch(queue, 0);
      atomicExch(queue + 1, 0);
    }
  }
}

// ------------------------------------------------------------------------------------------
// Host side: plans (one per batched solve: tensor maps built once) and launches
// ------------------------------------------------------------------------------------------
// Apply variants.  Every one computes the same split products; the choice only moves time.
enum { TCV_TWO_STAGE = 0, TCV_FUSED64 = 1, TCV_FUSED32 = 2, TCV_RESIDENT = 3, TCV_COUNT = 4 };

struct TCPlan {
  TCJob* d_fwd = nullptr;
  TCJob* d_bwd = nullptr;
  char* work = nullptr;   // Xt and Zt of every problem
  int njobs = 0, n = 0, kmax = 0;
  int prec = KPSB_P_TF32X3;
  bool bf = false;         // BF16 planes (BF16X3 / BF16X2)
  bool fused = false;      // single-launch apply (the variant is not the two-stage pair)
  int variant = 0;         // TCV_* chosen for this plan (autotuned, section below)
  bool ext_split = false;  // the caller writes the split planes (xt_ext)
  int* queue = nullptr;    // resident kernel: problem counter and finished-CTA counter (start at 0)
};

bool tc_plan_fused(const TCPlan* P) { return P && P->fused; }

int tc_plan_launches(const TCPlan* P) { return (P->ext_split ? 0 : 1) + (P->fused ? 1 : 2); }

static constexpr int S1_BN = 128, S1_STAGES = 3;
static constexpr int S2_BN = 64, S2_STAGES = 4;
// Stage 1 for n > 768: 256-column output tiles (one M = 128, N = 256 MMA per K step), half
// the CTAs and twice the work per prologue and epilogue (measured at n = 1024: -4 % BF16x3,
// -9 % TF32x2 per solve; slower at n = 512, where the CTAs no longer fill the GPU); the tile
// width does not change any element's accumulation order, so the bits are those of the
// 128-column tiles.
#ifndef KPSB_S1_BN_LARGE
#define KPSB_S1_BN_LARGE 256
#endif
static constexpr int S1L_BN = KPSB_S1_BN_LARGE;
static constexpr int s1l_stages(int fpl) { return S1L_BN == 128 ? S1_STAGES : (fpl == 2 ? 2 : 3); }
static inline bool s1_large(int n) { return n > 768; }

// Stage 2 where the two-stage kernel is the only variant for (n, precision), so its bits need
// not match the fused and resident kernels': BF16 planes, or TF32 with n > FUSED_MAX_N or n not
// a multiple of 128.  From n = 256 on it takes 128-column output tiles (half the operand bytes
// per MMA of 64-column tiles) and splits K into a fixed number of ranges, set by n alone so
// that up to about 128 CTAs share one problem (at most 8 ranges); the last CTA of a tile to
// finish adds the FP32 partial tiles in range order.  The split depends on n only, so a
// problem gives the same bits alone and in any batch.  Measured on one BF16x3 request (20
// outer steps): n = 1024 0.443 -> 0.387 s (split 2), n = 512 0.219 -> 0.173 s (split 8),
// n = 384 0.130 -> 0.113 s, n = 256 0.232 -> 0.166 s; 256-column tiles (two pipeline stages)
// and other splits were slower.
struct S2Shape {
  int bn, split;
};
static constexpr int S2W_BN = 128, S2W_STAGES = 3;
static S2Shape s2_shape(int n, bool bf) {
  const bool only_two_stage = bf || n % 128 != 0 || n > FUSED_MAX_N;
  if (!only_two_stage || n < 256) return {S2_BN, 1};
  const int tiles = ((n + 127) / 128) * ((n + S2W_BN - 1) / S2W_BN);
  return {S2W_BN, std::max(1, std::min(8, (128 + tiles / 2) / tiles))};
}
static size_t s2_split_bytes(int n, bool bf) {
  const S2Shape sh = s2_shape(n, bf);
  if (sh.split <= 1) return 0;
  const size_t tiles = (size_t)((n + 127) / 128) * ((n + sh.bn - 1) / sh.bn);
  return sizeof(float) * sh.split * tiles * 128 * sh.bn + sizeof(unsigned int) * tiles + 512;
}

template <int BN, int FPL>
static kpsb_status prepare_fused() {
  KPSB_TRY_CUDA(cudaFuncSetAttribute(tc_fused_kernel<BN, FPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     FCfg<BN, FPL>::SMEM));
  return KPSB_OK;
}

template <int BN, int FPL>
static kpsb_status launch_fused(const TCJob* jobs, int njobs, int n, cudaStream_t st) {
  dim3 grid((n + BN - 1) / BN, njobs);
  tc_fused_kernel<BN, FPL><<<grid, 192, FCfg<BN, FPL>::SMEM, st>>>(jobs);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

template <int FPL>
static kpsb_status prepare_resident() {
  KPSB_TRY_CUDA(cudaFuncSetAttribute(tc_resident_kernel<FPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     RCfg<FPL>::SMEM));
  return KPSB_OK;
}

template <int FPL>
static kpsb_status launch_resident(const TCJob* jobs, int njobs, int* queue, cudaStream_t st) {
  int dev = 0, sms = 0;
  KPSB_TRY_CUDA(cudaGetDevice(&dev));
  KPSB_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // persistent: one CTA per SM at most (fewer CTAs than problems measured slower: each
  // concurrent part's iteration waits for its own apply)
  const int grid = std::max(1, std::min(njobs, sms));
  tc_resident_kernel<FPL><<<grid, 192, RCfg<FPL>::SMEM, st>>>(jobs, njobs, queue);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

// Valid variants per size and precision (the autotuner picks among them; KPSB_TC_VARIANT pins
// one).  The fused and resident kernels are TF32 kernels for n a multiple of 128; the
// two-stage kernel runs every tensor-core precision and any n.
static bool variant_ok(int v, int n, int prec) {
  const bool tf = !prec_bf16(prec) && n % 128 == 0;
  switch (v) {
    case TCV_TWO_STAGE: return true;
    case TCV_FUSED64: return tf && n <= FUSED_MAX_N;
    case TCV_FUSED32: return tf && n <= FUSED_MAX_N;
    case TCV_RESIDENT: return tf && n == 128;
    default: return false;
  }
}

// Fused kernel up to n = FUSED_MAX_N (its TMEM would fit (R + 2) x BN columns up to n = 768, but
// from n = 512 on a fused CTA re-reads every stage-2 table for its 64 or 32 output columns, and
// the two-stage kernel with a K split is the better apply there).
static bool fused_ok(int n) { return n % 128 == 0 && n <= FUSED_MAX_N && (n / 128 + 2) * FUSED_BN <= 512; }


template <int BN, int STAGES, int STAGE, int FPL, bool BF>
static kpsb_status prepare_gemm() {
  using C = TCCfg<BN, STAGES, STAGE, FPL, BF>;
  KPSB_TRY_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<BN, STAGES, STAGE, FPL, BF>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
  return KPSB_OK;
}

static kpsb_status fill_job(TCJob& J, const KPJob& src, const TCTables* T, int transpose, bool bf, void* Xt,
                            int ldx, void* Zt) {
  const int n = src.n, k = src.k;
  J.X = src.X;
  J.Y = src.Y;
  J.Xt = Xt;
  J.Zt = Zt;
  J.n = n;
  J.k = k;
  J.ldz = T->ld2;
  J.ldx = ldx;
  J.active = src.active;
  J.Yf = src.yf;
  const cuuint64_t es = bf ? sizeof(__nv_bfloat16) : sizeof(float);
  const cuuint64_t l1 = (cuuint64_t)T->ld1, l2 = (cuuint64_t)T->ld2, lx = (cuuint64_t)ldx;
  const void* t1 = bf ? (const void*)(transpose ? T->B1t : T->B1f) : (const void*)(transpose ? T->T1t : T->T1f);
  const void* t2 = bf ? (const void*)(transpose ? T->B2t : T->B2f) : (const void*)(transpose ? T->T2t : T->T2f);
  {  // Xt: {n, n, 2}
    cuuint64_t d[3] = {(cuuint64_t)n, (cuuint64_t)n, 2};
    cuuint64_t s[2] = {es * lx, es * lx * n};
    KPSB_TRY(make_map(&J.m1A, Xt, 3, d, s, 128, bf));
  }
  cuuint64_t d1[4] = {(cuuint64_t)n, (cuuint64_t)n, 2, (cuuint64_t)k};
  cuuint64_t s1[3] = {es * l1, es * l1 * n, es * 2 * l1 * n};
  KPSB_TRY(make_map(&J.m1B, t1, 4, d1, s1, s1_large(n) ? S1L_BN : S1_BN, bf));  // T1: {n, n, 2, k}
  if (!bf && n % 128 == 0) {  // T1 with 64-, 32- and 128-row boxes (fused and resident kernels)
    KPSB_TRY(make_map(&J.m1F, t1, 4, d1, s1, 64));
    KPSB_TRY(make_map(&J.m1G, t1, 4, d1, s1, 32));
    KPSB_TRY(make_map(&J.m1R, t1, 4, d1, s1, 128));
  }
  cuuint64_t d2[3] = {(cuuint64_t)k * n, (cuuint64_t)n, 2};
  cuuint64_t s2[2] = {es * l2, es * l2 * n};
  KPSB_TRY(make_map(&J.m2A, t2, 3, d2, s2, 128, bf));    // T2: {k n, n, 2}
  KPSB_TRY(make_map(&J.m2B, Zt, 3, d2, s2, s2_shape(n, bf).bn, bf));  // Zt: {k n, n, 2}
  return KPSB_OK;
}

// ---- variant autotuner ----------------------------------------------------------------------
// Every variant computes each output element with the same sequence of MMAs (same K order,
// same order of the split products, same rounding of the intermediate), so all variants give
// the same bits and the choice only moves time.  The first plan of each (n, precision, k_max,
// batch-size bucket, split mode) times every valid variant on its own operands (two warm-up
// and four timed forward applies, CUDA events on the plan's stream, activity flags ignored)
// and keeps the fastest for the process.  A plan that is one of several concurrent parts of
// a batch (shared SMs) is ranked by SM time instead, duration x the CTAs the variant occupies
// (capped at the SM count): a variant that is faster alone only because it spreads over more
// SMs takes them from the other parts (measured on the 256-request step: a fused choice for one
// of four parts cost 12 % of the step).  KPSB_TC_VARIANT=v forces variant v where valid;
// KPSB_TUNE_LOG=1 prints the choices.
struct TuneKey {
  int n, prec, kmax, pbucket, ext, shared;
  bool operator<(const TuneKey& o) const {
    return std::tie(n, prec, kmax, pbucket, ext, shared) <
           std::tie(o.n, o.prec, o.kmax, o.pbucket, o.ext, o.shared);
  }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, int> g_tune;
static kpsb_status launch_variant(const TCPlan* P, const TCJob* jobs, int njobs, int variant, cudaStream_t st);

// CTAs a variant keeps busy at once, capped at the SM count.
static int variant_ctas(int variant, int n, int njobs, int kmax, int sms) {
  const long long tm = (n + 127) / 128;
  long long c;
  switch (variant) {
    case TCV_RESIDENT: c = njobs; break;
    case TCV_FUSED64: c = (long long)((n + 63) / 64) * njobs; break;
    case TCV_FUSED32: c = (long long)((n + 31) / 32) * njobs; break;
    default: c = tm * ((n + 127) / 128) * kmax * njobs; break;  // stage 1, the wider launch
  }
  return (int)std::max(1LL, std::min<long long>(c, sms));
}

static kpsb_status tune_variant(TCPlan* P, const std::vector<TCJob>& hf, bool shared, cudaStream_t st) {
  const int n = P->n;
  if (const char* f = getenv("KPSB_TC_VARIANT")) {
    const int v = atoi(f);
    if (variant_ok(v, n, P->prec)) { P->variant = v; return KPSB_OK; }
  }
  std::vector<int> cand;
  for (int v = 0; v < TCV_COUNT; ++v)
    if (variant_ok(v, n, P->prec)) cand.push_back(v);
  if (cand.size() == 1 || P->njobs == 0) { P->variant = cand[0]; return KPSB_OK; }
  int pb = 1;
  while (pb < P->njobs) pb <<= 1;
  const TuneKey key{n, P->prec, P->kmax, pb, P->ext_split ? 1 : 0, shared ? 1 : 0};
  std::lock_guard<std::mutex> lk(g_tune_mu);  // one tuner at a time; later plans reuse the choice
  auto it = g_tune.find(key);
  if (it != g_tune.end()) { P->variant = it->second; return KPSB_OK; }
  // operands as planned, without the activity flags (a new problem is not active yet)
  const int R = P->njobs;
  std::vector<TCJob> tj(hf);
  for (auto& J : tj) J.active = nullptr;
  TCJob* dj = nullptr;
  unsigned long long saved[2] = {0, 0};
  cudaEvent_t a = nullptr, b = nullptr;
  kpsb_status s = KPSB_OK;
  cudaError_t e = cudaMallocAsync((void**)&dj, sizeof(TCJob) * R, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dj, tj.data(), sizeof(TCJob) * R, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(saved, g_tc_work, sizeof(saved));  // tuning is not work
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  int dev = 0, sms = 1;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int best = cand[0];
  float best_ms = 0.f;
  constexpr int TUNE_REPS = 4;  // timed applies per candidate, after two warm-up applies
  for (size_t c = 0; c < cand.size() && e == cudaSuccess && s == KPSB_OK; ++c) {
    s = launch_variant(P, dj, R, cand[c], st);
    if (s == KPSB_OK) s = launch_variant(P, dj, R, cand[c], st);
    if (s == KPSB_OK) e = cudaEventRecord(a, st);
    for (int r = 0; r < TUNE_REPS && s == KPSB_OK && e == cudaSuccess; ++r) s = launch_variant(P, dj, R, cand[c], st);
    if (s == KPSB_OK && e == cudaSuccess) e = cudaEventRecord(b, st);
    if (s == KPSB_OK && e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (s == KPSB_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (shared) ms *= (float)variant_ctas(cand[c], n, R, P->kmax, sms);  // SM time
    if (s == KPSB_OK && e == cudaSuccess && (c == 0 || ms < best_ms)) {
      best = cand[c];
      best_ms = ms;
    }
    if (getenv("KPSB_TUNE_LOG") && e == cudaSuccess)
      fprintf(stderr, "[kpsb tune] n=%d prec=%d kmax=%d jobs<=%d shared=%d variant %d: %.3f %s\n", n, P->prec,
              P->kmax, pb, shared ? 1 : 0, cand[c], ms / TUNE_REPS, shared ? "SM-ms" : "ms");
  }
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc_work, saved, sizeof(saved));
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (dj) cudaFreeAsync(dj, st);
  if (s != KPSB_OK) return s;
  if (e != cudaSuccess) {
    set_error("tensor-core variant tuning: %s", cudaGetErrorString(e));
    return KPSB_ECUDA;
  }
  if (s == KPSB_OK) s = tc_check_error();
  if (s != KPSB_OK) return s;
  g_tune[key] = best;
  P->variant = best;
  return KPSB_OK;
}

kpsb_status tc_plan_create(kpsb_kp** kps, const KPJob* fwd_h, const KPJob* bwd_h, int njobs, int n,
                           int prec, cudaStream_t st, TCPlan** out, bool shared_sms) {
  KPSB_REQUIRE(tc_supported(n, prec), "no tensor-core kernel for n = %d, precision %d", n, prec);
  const bool bf = prec_bf16(prec);
  // a caller's split planes have leading dimension n and the plan's element type (the split
  // Bregman vector kernels write them in 32 x 32 tiles)
  for (int p = 0; p < njobs; ++p)
    KPSB_REQUIRE(!fwd_h[p].xt_ext || n % 32 == 0, "caller-split planes need n %% 32 == 0 (n = %d)", n);
  // kernel attributes are set here, before any graph capture that replays the applies
  KPSB_TRY((prepare_gemm<S1_BN, S1_STAGES, 1, 2, false>()));
  KPSB_TRY((prepare_gemm<S2_BN, S2_STAGES, 2, 2, false>()));
  KPSB_TRY((prepare_gemm<S1_BN, S1_STAGES, 1, 1, false>()));
  KPSB_TRY((prepare_gemm<S2_BN, S2_STAGES, 2, 1, false>()));
  KPSB_TRY((prepare_gemm<S1_BN, S1_STAGES, 1, 2, true>()));
  KPSB_TRY((prepare_gemm<S2_BN, S2_STAGES, 2, 2, true>()));
  KPSB_TRY((prepare_gemm<S1_BN, S1_STAGES, 1, 1, true>()));
  KPSB_TRY((prepare_gemm<S2_BN, S2_STAGES, 2, 1, true>()));
  KPSB_TRY((prepare_gemm<S1L_BN, s1l_stages(2), 1, 2, false>()));
  KPSB_TRY((prepare_gemm<S1L_BN, s1l_stages(1), 1, 1, false>()));
  KPSB_TRY((prepare_gemm<S1L_BN, s1l_stages(2), 1, 2, true>()));
  KPSB_TRY((prepare_gemm<S1L_BN, s1l_stages(1), 1, 1, true>()));
  KPSB_TRY((prepare_gemm<S2W_BN, S2W_STAGES, 2, 2, false>()));
  KPSB_TRY((prepare_gemm<S2W_BN, S2W_STAGES, 2, 1, false>()));
  KPSB_TRY((prepare_gemm<S2W_BN, S2W_STAGES, 2, 2, true>()));
  KPSB_TRY((prepare_gemm<S2W_BN, S2W_STAGES, 2, 1, true>()));
  KPSB_TRY((prepare_fused<FUSED_BN, 1>()));
  KPSB_TRY((prepare_fused<FUSED_BN, 2>()));
  KPSB_TRY((prepare_fused<32, 1>()));
  KPSB_TRY((prepare_fused<32, 2>()));
  KPSB_TRY(prepare_resident<1>());
  KPSB_TRY(prepare_resident<2>());
  TCPlan* P = new TCPlan();
  P->njobs = njobs;
  P->n = n;
  P->prec = prec;
  P->bf = bf;
  P->fused = !bf && fused_ok(n);  // the states carry split planes and FP32 outputs for a one-launch apply
  const size_t es = bf ? sizeof(__nv_bfloat16) : sizeof(float);
  const int ldx = pad8(n);
  std::vector<TCTables*> tabs(njobs);
  size_t bytes = 0;
  auto a256 = [](size_t x) { return (x + 255) / 256 * 256; };
  for (int p = 0; p < njobs; ++p) {
    kpsb_status s = tc_tables(kps[p], st, bf, &tabs[p]);
    if (s) {
      delete P;
      return s;
    }
    P->kmax = std::max(P->kmax, kps[p]->k);
    bytes += (fwd_h[p].xt_ext ? 0 : a256(es * 2 * n * ldx)) + a256(es * 2 * n * tabs[p]->ld2);
  }
  // stage-2 K split: FP32 partial tiles per problem (shared by its forward and transpose
  // applies, which never overlap) and one arrival counter per output tile, all zeroed once
  const S2Shape sh = s2_shape(n, bf);
  const size_t s2_tiles = (size_t)((n + 127) / 128) * ((n + sh.bn - 1) / sh.bn);
  const size_t part_bytes = sh.split > 1 ? a256(sizeof(float) * sh.split * s2_tiles * 128 * sh.bn) : 0;
  const size_t ctr_bytes = sh.split > 1 ? a256(sizeof(unsigned int) * s2_tiles * njobs) : 0;
  bytes += part_bytes * njobs + ctr_bytes;
  cudaError_t e = cudaMallocAsync((void**)&P->work, bytes + 2 * sizeof(TCJob) * njobs + 512, st);
  if (e != cudaSuccess) {
    delete P;
    set_error("tensor-core workspace: %s", cudaGetErrorString(e));
    return KPSB_ENOMEM;
  }
  std::vector<TCJob> hf(njobs), hb(njobs);
  char* q = P->work;
  unsigned int* ctrs = (unsigned int*)q;  // the counters first: one memset covers them
  q += ctr_bytes;
  if (ctr_bytes) e = cudaMemsetAsync(ctrs, 0, ctr_bytes, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(P->work, st);
    delete P;
    set_error("tensor-core workspace: %s", cudaGetErrorString(e));
    return KPSB_ECUDA;
  }
  P->ext_split = njobs > 0 && fwd_h[0].xt_ext != nullptr;
  for (int p = 0; p < njobs; ++p) {
    void* Xt = fwd_h[p].xt_ext;
    if (!Xt) {
      Xt = q;
      q += a256(es * 2 * n * ldx);
    }
    void* Zt = q;
    q += a256(es * 2 * n * tabs[p]->ld2);
    kpsb_status s = fill_job(hf[p], fwd_h[p], tabs[p], 0, bf, Xt, ldx, Zt);
    if (!s) s = fill_job(hb[p], bwd_h[p], tabs[p], 1, bf, Xt, ldx, Zt);
    float* part = nullptr;
    if (part_bytes) {
      part = (float*)q;
      q += part_bytes;
    }
    hf[p].part = hb[p].part = part;
    hf[p].tctr = hb[p].tctr = part ? ctrs + s2_tiles * p : nullptr;
    if (s) {
      cudaFreeAsync(P->work, st);
      delete P;
      return s;
    }
  }
  // Descriptors in decreasing k: the resident kernel's CTAs claim problems in this order, so
  // the largest problems start first and the last claims are the smallest (longest-first
  // scheduling evens out the CTAs' loads).  Each problem's arithmetic does not depend on
  // which CTA takes it; the other variants index descriptors by block and ignore the order.
  {
    std::vector<int> ord(njobs);
    for (int p = 0; p < njobs; ++p) ord[p] = p;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return hf[a].k > hf[b].k; });
    std::vector<TCJob> sf(njobs), sb(njobs);
    for (int p = 0; p < njobs; ++p) {
      sf[p] = hf[ord[p]];
      sb[p] = hb[ord[p]];
    }
    hf.swap(sf);
    hb.swap(sb);
  }
  char* jb = (char*)(((uintptr_t)q + 255) & ~(uintptr_t)255);
  P->d_fwd = (TCJob*)jb;
  P->d_bwd = P->d_fwd + njobs;
  P->queue = (int*)(P->d_bwd + njobs);
  e = cudaMemsetAsync(P->queue, 0, 2 * sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_fwd, hf.data(), sizeof(TCJob) * njobs, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_bwd, hb.data(), sizeof(TCJob) * njobs, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host job arrays go out of scope
  if (e != cudaSuccess) {
    cudaFreeAsync(P->work, st);
    delete P;
    set_error("tensor-core plan upload: %s", cudaGetErrorString(e));
    return KPSB_ECUDA;
  }
  kpsb_status ts = tune_variant(P, hf, shared_sms, st);
  if (ts != KPSB_OK) {
    tc_plan_free(P, st);
    return ts;
  }
  P->fused = P->variant != TCV_TWO_STAGE;
  *out = P;
  return KPSB_OK;
}

void tc_plan_free(TCPlan* P, cudaStream_t st) {
  if (!P) return;
  if (P->work) cudaFreeAsync(P->work, st);
  delete P;
}

template <int BN, int STAGES, int STAGE, int FPL, bool BF>
static kpsb_status launch_gemm(const TCJob* jobs, int njobs, int n, int kmax, cudaStream_t st, int split = 1) {
  using C = TCCfg<BN, STAGES, STAGE, FPL, BF>;
  const int tiles_m = (n + 127) / 128, tiles_n = (n + BN - 1) / BN;
  dim3 grid(tiles_m * tiles_n, STAGE == 1 ? kmax : split, njobs);
  tc_gemm_kernel<BN, STAGES, STAGE, FPL, BF><<<grid, 128, C::SMEM, st>>>(jobs, tiles_m);
  KPSB_CHECK_LAUNCH();
  return KPSB_OK;
}

template <int FPL, bool BF>
static kpsb_status launch_two_stage(const TCJob* jobs, int njobs, int n, int kmax, cudaStream_t st) {
  if (s1_large(n)) KPSB_TRY((launch_gemm<S1L_BN, s1l_stages(FPL), 1, FPL, BF>(jobs, njobs, n, kmax, st)));
  else KPSB_TRY((launch_gemm<S1_BN, S1_STAGES, 1, FPL, BF>(jobs, njobs, n, kmax, st)));
  const S2Shape sh = s2_shape(n, BF);
  if (sh.bn == S2W_BN) KPSB_TRY((launch_gemm<S2W_BN, S2W_STAGES, 2, FPL, BF>(jobs, njobs, n, kmax, st, sh.split)));
  else KPSB_TRY((launch_gemm<S2_BN, S2_STAGES, 2, FPL, BF>(jobs, njobs, n, kmax, st)));
  return KPSB_OK;
}

static kpsb_status launch_variant(const TCPlan* P, const TCJob* jobs, int njobs, int variant, cudaStream_t st) {
  const int n = P->n;
  const bool two = prec_fpl(P->prec) == 2;
  switch (variant) {
    case TCV_RESIDENT: return two ? launch_resident<2>(jobs, njobs, P->queue, st)
                                  : launch_resident<1>(jobs, njobs, P->queue, st);
    case TCV_FUSED64: return two ? launch_fused<64, 2>(jobs, njobs, n, st) : launch_fused<64, 1>(jobs, njobs, n, st);
    case TCV_FUSED32: return two ? launch_fused<32, 2>(jobs, njobs, n, st) : launch_fused<32, 1>(jobs, njobs, n, st);
    default: break;
  }
  if (P->bf) return two ? launch_two_stage<2, true>(jobs, njobs, n, P->kmax, st)
                        : launch_two_stage<1, true>(jobs, njobs, n, P->kmax, st);
  return two ? launch_two_stage<2, false>(jobs, njobs, n, P->kmax, st)
             : launch_two_stage<1, false>(jobs, njobs, n, P->kmax, st);
}

kpsb_status tc_plan_apply(TCPlan* P, int transpose, cudaStream_t st) {
  const TCJob* jobs = transpose ? P->d_bwd : P->d_fwd;
  const int n = P->n;
  if (!P->ext_split) {
    const int t = (n + 31) / 32;
    dim3 gs(t * t, P->njobs);
    if (P->bf) tc_split_kernel<__nv_bfloat16><<<gs, 256, 0, st>>>(jobs);
    else tc_split_kernel<float><<<gs, 256, 0, st>>>(jobs);
    KPSB_CHECK_LAUNCH();
  }
  return launch_variant(P, jobs, P->njobs, P->variant, st);
}

kpsb_status tc_work(unsigned long long* out, bool reset) {
  if (reset) {
    const unsigned long long z[2] = {0, 0};
    KPSB_TRY_CUDA(cudaMemcpyToSymbol(g_tc_work, z, sizeof(z)));
  }
  if (out) KPSB_TRY_CUDA(cudaMemcpyFromSymbol(out, g_tc_work, 2 * sizeof(unsigned long long)));
  return KPSB_OK;
}

kpsb_status tc_check_error() {
  int h = 0;
  KPSB_TRY_CUDA(cudaMemcpyFromSymbol(&h, g_tc_error, sizeof(int)));
  if (h) {
    int z = 0;
    cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
    set_error("tensor-core GEMM: a pipeline wait timed out");
    return KPSB_ETIMEOUT;
  }
  return KPSB_OK;
}

// Single apply through a temporary plan (kp_apply_dev).
kpsb_status tc_apply_batch(kpsb_kp** kps, const KPJob* jobs_d, const KPJob* jobs_h, int njobs, int n,
                           int kmax, int transpose, int prec, cudaStream_t st) {
  (void)jobs_d;
  (void)kmax;
  KPSB_REQUIRE(prec_is_tc(prec), "precision %d has no tensor-core kernel", prec);
  TCPlan* P = nullptr;
  KPSB_TRY(tc_plan_create(kps, jobs_h, jobs_h, njobs, n, prec, st, &P));
  kpsb_status s = tc_plan_apply(P, transpose, st);
  cudaError_t e = cudaStreamSynchronize(st);
  tc_plan_free(P, st);
  if (s == KPSB_OK && e != cudaSuccess) {
    set_error("tensor-core apply: %s", cudaGetErrorString(e));
    s = KPSB_ECUDA;
  }
  if (s == KPSB_OK) s = tc_check_error();
  return s;
}

}  // namespace kpsb

using namespace kpsb;

extern "C" int kpsb_tuned_variants(int* rows, int max_rows) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  int i = 0;
  for (const auto& kv : g_tune) {
    if (rows && i < max_rows) {
      int* r = rows + 7 * i;
      r[0] = kv.first.n;
      r[1] = kv.first.prec;
      r[2] = kv.first.kmax;
      r[3] = kv.first.pbucket;
      r[4] = kv.first.ext;
      r[5] = kv.first.shared;
      r[6] = kv.second;
    }
    ++i;
  }
  return i;
}

extern "C" kpsb_status kpsb_wait_selftest(unsigned int limit_us) {
  clear_error();
  KPSB_REQUIRE(limit_us >= 1 && limit_us <= 1000000u, "limit_us must be in [1, 1000000] (got %u)", limit_us);
  int dev = 0, khz = 0;
  KPSB_TRY_CUDA(cudaGetDevice(&dev));
  KPSB_TRY_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
  if (khz <= 0) khz = 2000000;
  int* d = nullptr;
  KPSB_TRY_CUDA(cudaMalloc((void**)&d, sizeof(int)));
  tc_wait_selftest_kernel<<<1, 32>>>((long long)limit_us * (khz / 1000), d);
  count_launch();
  cudaError_t e = cudaGetLastError();
  int h = -1;
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    set_error("kpsb_wait_selftest: %s", cudaGetErrorString(e));
    return KPSB_ECUDA;
  }
  kpsb_status s = tc_check_error();  // KPSB_ETIMEOUT once the wait has run out
  if (s == KPSB_OK && h != 1) {
    set_error("kpsb_wait_selftest: the wait neither completed nor recorded a time-out");
    return KPSB_ECUDA;
  }
  return s;
}

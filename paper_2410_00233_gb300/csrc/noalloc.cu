// R(A) block apply that allocates nothing: the same reduce / expand kernels as
// kp_ra_apply_dev, with their scratch (per-tile partial sums, mixed tap weights and the
// last-block counters) in a fixed-size array that lives in device memory for as long as
// the library is loaded.
//
// Who needs it: callers that must not allocate device memory during a call.  A real-time
// imaging loop cannot afford cudaMalloc/cudaFree, which may synchronise the whole device
// and take milliseconds; a host program that hands all device memory to its own pool at
// start-up, or runs under a strict memory budget, has no allocator to spare for a
// library.  Those callers pass their own inputs and outputs, and the scratch comes from
// here.
#include "kpsb_internal.cuh"

namespace kpsb {

// 4 MiB: enough for n <= 512 with up to 60 vectors per call, or n = 1024 with up to 15.
static constexpr size_t NOALLOC_SCRATCH_BYTES = 4u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on the device that owns `st`.  In host code
// g_noalloc_scratch names a host-side shadow, not device memory, so only the address that
// cudaGetSymbolAddress returns may be handed to a kernel.  The address is looked up on every
// call (a table lookup once the module is loaded), so it follows the current context even
// after a cudaDeviceReset.  The first lookup on a device loads the module there, which is
// why the first call belongs before any stream capture.
static kpsb_status noalloc_scratch(cudaStream_t st, void** out) {
  int dev = 0;
  KPSB_TRY_CUDA(cudaGetDevice(&dev));
  if (st) {
    int sdev = -1;
    KPSB_TRY_CUDA(cudaStreamGetDevice(st, &sdev));
    KPSB_REQUIRE(sdev == dev,
                 "kp_ra_apply_noalloc_dev: the stream belongs to device %d but device %d is current",
                 sdev, dev);
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    set_error("cudaGetSymbolAddress of the scratch array failed on device %d: %s", dev,
              cudaGetErrorString(e));
    return KPSB_ECUDA;
  }
  *out = p;
  return KPSB_OK;
}

}  // namespace kpsb

using namespace kpsb;

extern "C" kpsb_status kp_ra_apply_noalloc_dev(const float* psf, int s0, int s1, int n, int bc,
                                               const float* V, int ldv, int nb, float* U, int ldu,
                                               int transpose, void* stream) {
  clear_error();
  KPSB_TRY(ra_check(s0, s1, n, bc));
  KPSB_REQUIRE(psf && V && U, "null pointer");
  KPSB_REQUIRE(nb >= 1 && ldv >= n * n && ldu >= n * n, "bad block shape nb=%d ldv=%d ldu=%d", nb,
               ldv, ldu);
  const int s_exp = transpose ? s0 : s1;
  const size_t need = ra_scratch_bytes(n, nb, s_exp);
  KPSB_REQUIRE(need <= NOALLOC_SCRATCH_BYTES,
               "kp_ra_apply_noalloc_dev: n=%d, nb=%d, s=%d needs %zu bytes of scratch, more than "
               "the fixed %zu (use fewer vectors per call, or kp_ra_apply_dev)",
               n, nb, s_exp, need, (size_t)NOALLOC_SCRATCH_BYTES);
  cudaStream_t st = (cudaStream_t)stream;
  void* base = nullptr;
  KPSB_TRY(noalloc_scratch(st, &base));
  RAScratch scr = ra_scratch_carve(base, n, nb, s_exp);
  // the array keeps the previous call's contents: the counters must start at zero
  KPSB_TRY_CUDA(cudaMemsetAsync(scr.counters, 0, sizeof(unsigned int) * nb, st));
  return ra_apply(psf, s0, s1, n, bc, V, ldv, nb, U, ldu, transpose, nullptr, 0, nullptr, 0.f,
                  nullptr, scr, st);
}

// Tensor-core (tcgen05) Kronecker-sum GEMMs: placeholder until the kernels land.
#include "kpsb_internal.cuh"

namespace kpsb {

struct TCTables {};

bool tc_supported(int, int) { return false; }

void tc_free(TCTables* t) { delete t; }

kpsb_status tc_apply_batch(kpsb_kp**, const KPJob*, const KPJob*, int, int, int, int, int,
                           cudaStream_t) {
  set_error("tensor-core KP GEMM not available in this build");
  return KPSB_EINVAL;
}

}  // namespace kpsb

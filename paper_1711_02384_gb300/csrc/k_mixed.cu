// Mixed-precision path (FP32 site contraction, split-FP16 tensor-core projection).
#include "lhc_internal.h"

namespace lhc {

int run_slice_mixed(lhc_ctx ctx, const SliceJob &job, const int *k, int nq, const int r[4], int sign,
                    cudaStream_t st) {
  (void)ctx; (void)job; (void)k; (void)nq; (void)r; (void)sign; (void)st;
  set_error("mixed precision path not built yet");
  return LHC_EINVAL;
}

}  // namespace lhc

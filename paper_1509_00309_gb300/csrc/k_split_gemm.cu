// Split-precision dense x dense tile products on the tcgen05 tensor cores (placeholder until
// the kernel lands).
#include "clr_internal.h"

namespace clr {

int split_gemm_dd(const SplitGemmArgs& a, cudaStream_t st, std::string* why) {
  (void)a;
  (void)st;
  if (why) *why = "split-precision tensor-core path not built";
  return CLR_ENOTSUP;
}

}  // namespace clr

// k_eval_tc.cu -- tensor-core evaluation (placeholder until the tcgen05 kernel lands).
#include "ubqp_internal.cuh"

namespace ubqp {
size_t eval_tc_workspace(const ubqp_q*, int64_t) { return 0; }
cudaError_t launch_eval_tc(const ubqp_q*, const uint64_t*, int64_t, int64_t*, void*, size_t,
                           cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace ubqp

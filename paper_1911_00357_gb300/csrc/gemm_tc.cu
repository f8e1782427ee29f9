// tcgen05 BF16 GEMM (placeholder: shapes route to the SIMT kernel until it lands).
#include "gemm.cuh"

namespace ddppo {
bool gemm_tc_supported(const GemmDesc&) { return false; }
int gemm_tc(const GemmDesc&, const GemmWorkspace&, cudaStream_t) {
  set_error("tcgen05 GEMM not built");
  return DDPPO_E_CONFIG;
}
}  // namespace ddppo

// Tensor-core product (placeholder until the tcgen05 kernel lands).
#include "symnmf_internal.h"
namespace symnmf {
bool tc_supported(int, int) { return false; }
cudaError_t launch_prod_tc(const ProdArgs &, cudaStream_t, int) { return cudaErrorNotSupported; }
}  // namespace symnmf

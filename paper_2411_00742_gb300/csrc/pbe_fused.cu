// Fused path: placeholder until the persistent kernels land.
#include "pbe_internal.h"

namespace pbe {
bool fused_supported(const pbe_grid*) { return false; }
cudaError_t launch_fused_solve(pbe_grid*, int) { return cudaErrorNotSupported; }
}  // namespace pbe

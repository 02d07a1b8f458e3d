// compose_batched_c128.cu -- the batched composition kernel (compose_batched.cuh), c128.
#include "compose_batched.cuh"

namespace pauli {
cudaError_t compose_batched_c128(const cb::ComposeTable& tab, int batch, int n_items, int scale_exp, cudaStream_t s) {
  return cb::launch_t<xd::ArC128>(tab, batch, n_items, scale_exp, s);
}
}  // namespace pauli

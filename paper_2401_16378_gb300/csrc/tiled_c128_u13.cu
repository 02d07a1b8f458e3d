// tiled_c128_u13.cu -- two-stage tiled decomposition, complex128, 8192-element units.
#include "tiled_impl.cuh"

namespace pauli {
cudaError_t tiled_launch_c128_u13(const void* G, int N, int count, void* out, cudaStream_t st) {
  return tiled::launch_tiled_n<13, xd::ArC128>(G, N, count, out, st);
}
}  // namespace pauli

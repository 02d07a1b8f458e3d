// tiled_c64_u12.cu -- two-stage tiled decomposition, complex64, 4096-element units.
#include "tiled_impl.cuh"

namespace pauli {
cudaError_t tiled_launch_c64_u12(const void* G, int N, int count, void* out, cudaStream_t st) {
  return tiled::launch_tiled_n<12, xd::ArC64>(G, N, count, out, st);
}
}  // namespace pauli

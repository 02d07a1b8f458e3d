// tiled_real_r4.cu -- two-stage tiled decomposition of real (float64) matrices, 16 elements per
// consumer thread.
#include "tiled_impl.cuh"
#include "xordiag_real.cuh"

namespace pauli {
cudaError_t tiled_launch_real_r4(const void* G, int N, int count, void* out, cudaStream_t st) {
  return tiled::launch_tiled_n<4, xd::ArR128>(G, N, count, out, st);
}
}  // namespace pauli

// tiled_c128_r3.cu -- two-stage tiled decomposition, complex128, 8 elements per consumer thread
// (complex and real-part outputs).
#include "tiled_impl.cuh"

namespace pauli {
cudaError_t tiled_launch_c128_r3(const void* G, int N, int count, void* out, cudaStream_t st) {
  return tiled::launch_tiled_n<3, xd::ArC128>(G, N, count, out, st);
}
cudaError_t tiled_launch_re_c128_r3(const void* G, int N, int count, void* out, cudaStream_t st) {
  return tiled::launch_tiled_n<3, xd::ReOut<xd::ArC128>>(G, N, count, out, st);
}
}  // namespace pauli

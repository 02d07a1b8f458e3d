// tiled_c64_r3.cu -- two-stage tiled decomposition, complex64, 8 elements per consumer thread
// (complex and real-part outputs).
#include "tiled_impl.cuh"

namespace pauli {
cudaError_t tiled_launch_c64_r3(const void* G, int N, int count, void* out, cudaStream_t st) {
  return tiled::launch_tiled_n<3, xd::ArC64T>(G, N, count, out, st);
}
cudaError_t tiled_launch_re_c64_r3(const void* G, int N, int count, void* out, cudaStream_t st) {
  return tiled::launch_tiled_n<3, xd::ReOut<xd::ArC64T>>(G, N, count, out, st);
}
}  // namespace pauli

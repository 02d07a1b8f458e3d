// tiled_c128_r4.cu -- two-stage tiled decomposition, complex128, 16 elements per consumer thread
// (complex and real-part outputs).
#include "tiled_impl.cuh"

namespace pauli {
cudaError_t tiled_launch_c128_r4(const void* G, int N, int count, void* out, cudaStream_t st) {
  return tiled::launch_tiled_n<4, xd::ArC128>(G, N, count, out, st);
}
cudaError_t tiled_launch_re_c128_r4(const void* G, int N, int count, void* out, cudaStream_t st) {
  return tiled::launch_tiled_n<4, xd::ReOut<xd::ArC128>>(G, N, count, out, st);
}
size_t tiled_workspace_bytes(int N) {
  switch (N) {
    case 12: return tiled::Geo<12>::kWorkspace;
    case 13: return tiled::Geo<13>::kWorkspace;
    case 14: return tiled::Geo<14>::kWorkspace;
    default: return 0;
  }
}
size_t tiled_workspace_max_bytes() {
  size_t m = 0;
  for (int N = 12; N <= 14; ++N) m = tiled_workspace_bytes(N) > m ? tiled_workspace_bytes(N) : m;
  return m;
}
}  // namespace pauli

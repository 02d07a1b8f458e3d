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
size_t twostage_workspace_bytes_c128(int N);
size_t tiled_workspace_bytes(int N) {
  size_t b = 0;
  switch (N) {
    case 12: b = tiled::Geo<12>::kWorkspace; break;
    case 13: b = tiled::Geo<13>::kWorkspace; break;
    case 14: b = tiled::Geo<14>::kWorkspace; break;
    default: return 0;
  }
  const size_t t = twostage_workspace_bytes_c128(N);
  return t > b ? t : b;
}
size_t tiled_workspace_max_bytes() {
  size_t m = 0;
  for (int N = 12; N <= 14; ++N) m = tiled_workspace_bytes(N) > m ? tiled_workspace_bytes(N) : m;
  return m;
}
}  // namespace pauli

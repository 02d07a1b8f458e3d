// twostage_c64.cu -- the warp-independent two-stage decomposition (twostage_impl.cuh), c64,
// complex and real-part outputs.
#include "twostage_impl.cuh"

namespace pauli {
cudaError_t twostage_launch_c64(const void* G, int N, int count, void* out, cudaStream_t st) {
  return ts::launch_n<xd::ArC64X>(G, N, count, out, st);
}
cudaError_t twostage_launch_upper_c64(const void* G, int N, int count, void* out, cudaStream_t st) {
  return ts::launch_upper_n<xd::ReOut<xd::ArC64X>>(G, N, count, out, st);
}
cudaError_t twostage_launch_xhi_c64(const void* L, int N, int k, uint32_t x_hi, void* out, cudaStream_t st) {
  return ts::launch_xhi_n<xd::ArC64X>(L, N, k, x_hi, out, st);
}
cudaError_t twostage_launch_re_c64(const void* G, int N, int count, void* out, cudaStream_t st) {
  return ts::launch_n<xd::ReOut<xd::ArC64X>>(G, N, count, out, st);
}
size_t twostage_workspace_bytes_c64(int N) {
  switch (N) {
    case 12: return ts::Geo<12, ts::kScratchEntry<xd::ArC64X>>::kWorkspace;
    case 13: return ts::Geo<13, ts::kScratchEntry<xd::ArC64X>>::kWorkspace;
    case 14: return ts::Geo<14, ts::kScratchEntry<xd::ArC64X>>::kWorkspace;
    default: return 0;
  }
}
}  // namespace pauli

// xordiag_herm_c64.cu -- c64 decomposition of a Hermitian G from its upper triangle.
#include "xordiag_herm.cuh"

namespace pauli {
cudaError_t xordiag_herm_upper_c64(int N, const void* in, long long count, void* out, cudaStream_t st) {
  return xh::dispatch_herm<xd::ReOut<xd::ArC64>>(N, in, count, out, st);
}
}  // namespace pauli

// xordiag_fused_c64_norm.cu -- c64 decomposition that also sums w_n |c_n|^2 of the
// coefficients it stores (one partial per work unit).
#include "xordiag_fused.cuh"

namespace pauli {
cudaError_t fused_decompose_norm_c64(int N, bool unit4096, const void* G, long long count, void* out,
                                      const void* w, double* partial, cudaStream_t st) {
  return xf::by_n<xd::ArC64, false, xd::NormOutEpi>(N, unit4096, G, count, 0, out, xd::EpiArgs{w, nullptr, partial},
                                                    st);
}
}  // namespace pauli

// xordiag_fused_c64_weighted.cu -- c64 composition of the weighted coefficients g w_n c_n.
#include "xordiag_fused.cuh"

namespace pauli {
cudaError_t fused_compose_weighted_c64(int N, bool unit4096, const void* c, long long count, int scale_exp,
                                         void* G, const void* w, const void* g, cudaStream_t st) {
  return xf::by_n<xd::ArC64, true, xd::WeightInEpi>(N, unit4096, c, count, scale_exp, G, xd::EpiArgs{w, g, nullptr},
                                                    st);
}
}  // namespace pauli

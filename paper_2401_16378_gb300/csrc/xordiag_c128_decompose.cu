// xordiag_c128_decompose.cu -- c128 decomposition instantiations of the XOR-diagonal kernels.
#include "xordiag_kernels.cuh"

namespace pauli {

cudaError_t xordiag_c128_decompose(int variant, int N, const void* in, long long count, int scale_exp, void* out,
                 cudaStream_t st) {
  return xk::dispatch_variant<xd::ArC128, false>(variant, N, in, count, scale_exp, out, st);
}

}  // namespace pauli

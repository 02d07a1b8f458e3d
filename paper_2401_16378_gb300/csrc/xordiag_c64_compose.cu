// xordiag_c64_compose.cu -- c64 composition instantiations of the XOR-diagonal kernels.
#include "xordiag_kernels.cuh"

namespace pauli {

cudaError_t xordiag_c64_compose(int variant, int N, const void* in, long long count, int scale_exp, void* out,
                 cudaStream_t st) {
  return xk::dispatch_variant<xd::ArC64, true>(variant, N, in, count, scale_exp, out, st);
}

}  // namespace pauli

// xordiag_re_c64.cu -- c64 real-part (Hermitian) decompositions of the single-pass XOR-diagonal
// kernels, 16 elements per thread: 8192-element units on one 512-thread CTA per SM, or
// 4096-element units on two 256-thread CTAs per SM (always at N = 6).
#include "xordiag_kernels.cuh"

namespace pauli {

cudaError_t xordiag_re_decompose_c64(int N, const void* in, long long count, void* out, cudaStream_t st,
                                     bool unit4096) {
  using AR = xd::ReOut<xd::ArC64>;
  if (unit4096 || N == 6) return xk::dispatch_shape<12, 4, AR, false>(N, in, count, 0, out, st);
  return xk::dispatch_shape<13, 4, AR, false>(N, in, count, 0, out, st);
}

}  // namespace pauli

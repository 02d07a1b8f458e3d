// xordiag_re_c64.cu -- c64 real-part (Hermitian) decompositions of the single-pass XOR-diagonal
// kernels: 8192-element units of 16 elements per thread (4096-element units at N = 6).
#include "xordiag_kernels.cuh"

namespace pauli {

cudaError_t xordiag_re_decompose_c64(int N, const void* in, long long count, void* out, cudaStream_t st) {
  using AR = xd::ReOut<xd::ArC64>;
  if (N == 6) return xk::launch_one<12, 4, 6, AR, false>(in, count, 0, out, st);
  return xk::dispatch_shape<13, 4, AR, false>(N, in, count, 0, out, st);
}

}  // namespace pauli

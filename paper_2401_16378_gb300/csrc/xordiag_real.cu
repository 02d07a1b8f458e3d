// xordiag_real.cu -- decompositions of real (float64) matrices with the single-pass XOR-diagonal
// kernels, 16 elements per thread: 8192-element units, or 4096-element units (always at N = 6).
#include "xordiag_kernels.cuh"
#include "xordiag_real.cuh"

namespace pauli {

cudaError_t xordiag_real_decompose(int N, const void* in, long long count, void* out, cudaStream_t st,
                                   bool unit4096) {
  using AR = xd::ArR128;
  if (unit4096 || N == 6) return xk::dispatch_shape<12, 4, AR, false>(N, in, count, 0, out, st);
  return xk::dispatch_shape<13, 4, AR, false>(N, in, count, 0, out, st);
}

}  // namespace pauli

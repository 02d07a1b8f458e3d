// fused.cu -- host side of the fused forms of the adjoint workload's step:
//   forward:  c = decompose(G) and L = sum_k sum_n w_n |c_kn|^2 in one pass over G
//             (the decomposition kernel accumulates L over the coefficients it stores);
//   backward: dL/dG = 2^-N compose(2 g w c) in one pass over c (the composition kernel
//             multiplies each loaded c_n by g w_n; the factor 2 is the exact scale 2^(1-N)).
// Fused single-pass kernels cover N = 6..12 (xordiag_fused_*.cu); other N take the unfused
// kernels in sequence (the decomposition and the norm; the plain composition with weights for
// N < 6) or report cudaErrorNotSupported (weighted composition above N = 12).
#include "kernels.h"
#include "workspace.h"

namespace pauli {

cudaError_t fused_decompose_norm_c128(int, bool, const void*, long long, void*, const void*, double*, cudaStream_t);
cudaError_t fused_decompose_norm_c64(int, bool, const void*, long long, void*, const void*, double*, cudaStream_t);
cudaError_t fused_compose_weighted_c128(int, bool, const void*, long long, int, void*, const void*, const void*,
                                        cudaStream_t);
cudaError_t fused_compose_weighted_c64(int, bool, const void*, long long, int, void*, const void*, const void*,
                                       cudaStream_t);

namespace {

// 4096-element units where the tuned (or built-in) shape for this call is a 4096-element one.
bool use_unit4096(int N, bool c64, bool compose, long long count) {
  if (N == 6) return true;
  if (N >= 12) return false;
  const int v = xordiag_get_variant(N, c64, compose, count > 1);
  return v == kVariantUnit12 || v == kVariantUnit12x8;
}

}  // namespace

cudaError_t launch_decompose_norm(const void* G, int N, long long count, bool c64, void* out, const void* w,
                                  void* loss, int method, cudaStream_t st) {
  cudaError_t e;
  if (method != 1 && N >= 6 && N <= 12) {  // XOR-diagonal, fused
    const bool u4 = use_unit4096(N, c64, false, count);
    const unsigned long long units = ((unsigned long long)count << (2 * N)) >> (u4 ? 12 : 13);
    void* ws = nullptr;
    if ((e = stream_workspace(kWorkspaceNorm, st, units * sizeof(double), kNormWorkspaceReserve, 0, &ws)) != cudaSuccess) return e;
    double* partial = static_cast<double*>(ws);
    e = c64 ? fused_decompose_norm_c64(N, u4, G, count, out, w, partial, st)
            : fused_decompose_norm_c128(N, u4, G, count, out, w, partial, st);
    if (e != cudaSuccess) return e;
    return launch_norm_final(partial, (long long)units, c64, loss, st);
  }
  e = (method == 1 || !xordiag_supported(N)) ? launch_plain_decompose(G, N, count, c64, out, st)
                                             : launch_xordiag(G, N, count, c64, false, 0, out, st);
  if (e != cudaSuccess) return e;
  return launch_weighted_norm(out, N, count, c64, w, loss, st);
}

cudaError_t launch_compose_weighted(const void* c, int N, long long count, bool c64, const void* w, const void* g,
                                    int scale_exp, void* G, cudaStream_t st) {
  if (N < 6) return launch_plain_compose(c, N, count, c64, scale_exp, G, st, w, g);
  if (N > 12) return cudaErrorNotSupported;
  const bool u4 = use_unit4096(N, c64, true, count);
  return c64 ? fused_compose_weighted_c64(N, u4, c, count, scale_exp, G, w, g, st)
             : fused_compose_weighted_c128(N, u4, c, count, scale_exp, G, w, g, st);
}

}  // namespace pauli

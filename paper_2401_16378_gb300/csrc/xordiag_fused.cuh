// xordiag_fused.cuh -- dispatch over N of the single-pass kernels with fused work (included by
// the per-dtype, per-direction translation units xordiag_fused_*.cu).
#pragma once
#include "xordiag_kernels.cuh"

namespace pauli {
namespace xf {

template <int UB, int N, class AR, bool COMPOSE, class EPI>
cudaError_t one(const void* in, long long count, int scale_exp, void* out, const xd::EpiArgs& ea, cudaStream_t st) {
  return xk::launch_one<UB, 4, N, AR, COMPOSE, EPI>(in, count, scale_exp, out, st, ea);
}

// N 6..11 on 4096-element units (two 256-thread CTAs per SM), or N 7..12 on 8192-element units
// (one 512-thread CTA per SM); 16 elements per thread.
template <class AR, bool COMPOSE, class EPI>
cudaError_t by_n(int N, bool unit4096, const void* in, long long count, int scale_exp, void* out,
                 const xd::EpiArgs& ea, cudaStream_t st) {
  if (unit4096 || N == 6) {
    switch (N) {
      case 6: return one<12, 6, AR, COMPOSE, EPI>(in, count, scale_exp, out, ea, st);
      case 7: return one<12, 7, AR, COMPOSE, EPI>(in, count, scale_exp, out, ea, st);
      case 8: return one<12, 8, AR, COMPOSE, EPI>(in, count, scale_exp, out, ea, st);
      case 9: return one<12, 9, AR, COMPOSE, EPI>(in, count, scale_exp, out, ea, st);
      case 10: return one<12, 10, AR, COMPOSE, EPI>(in, count, scale_exp, out, ea, st);
      case 11: return one<12, 11, AR, COMPOSE, EPI>(in, count, scale_exp, out, ea, st);
      default: return cudaErrorNotSupported;
    }
  }
  switch (N) {
    case 7: return one<13, 7, AR, COMPOSE, EPI>(in, count, scale_exp, out, ea, st);
    case 8: return one<13, 8, AR, COMPOSE, EPI>(in, count, scale_exp, out, ea, st);
    case 9: return one<13, 9, AR, COMPOSE, EPI>(in, count, scale_exp, out, ea, st);
    case 10: return one<13, 10, AR, COMPOSE, EPI>(in, count, scale_exp, out, ea, st);
    case 11: return one<13, 11, AR, COMPOSE, EPI>(in, count, scale_exp, out, ea, st);
    case 12: return one<13, 12, AR, COMPOSE, EPI>(in, count, scale_exp, out, ea, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace xf
}  // namespace pauli

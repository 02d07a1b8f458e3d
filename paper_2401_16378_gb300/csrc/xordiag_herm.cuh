// xordiag_herm.cuh -- decomposition of a Hermitian G read from its upper triangle (real
// coefficients), N = 7..12, one 512-thread CTA per unit of 8192 elements (included by
// xordiag_herm_c128.cu and xordiag_herm_c64.cu). The unit algorithm is run_unit_herm in
// xordiag_impl.cuh.
#pragma once
#include "xordiag_kernels.cuh"

namespace pauli {
namespace xh {
using namespace xd;

// A unit is 2^KH classes x 2^(N-1) rows (KH = 14 - N); the classes of unit 0 of each matrix
// (x < 2^KH: the diagonal and classes of different top bits) take two full-row units with the
// lower triangle read through its mirror instead.
template <int N, class AR>
__global__ void __launch_bounds__(Unit<13, 4>::kThreads, 1)
    xordiag_herm_kernel(const void* __restrict__ in, void* __restrict__ out, unsigned long long units,
                        unsigned long long ahead) {
  constexpr int UB = 13, RB = 4;
  constexpr int KH = UB - (N - 1), KR = UB - N;
  constexpr uint32_t D = 1u << N;
  extern __shared__ __align__(16) uint4 xbuf[];
  __shared__ uint32_t smax[1 << KH];
  const uint32_t t = threadIdx.x;
  const uint32_t xaddr = (uint32_t)__cvta_generic_to_shared(xbuf);
  const unsigned long long upm = D >> KH;  // units per matrix
  const unsigned long long unit = blockIdx.x;
  const unsigned long long base = (unit / upm) * (unsigned long long)D * D;
  const uint32_t xb = (uint32_t)(unit % upm) << KH;
  const unsigned long long nu = unit + ahead;
  auto prefetch_ahead = [&]() {
    if (nu < units && nu % upm != 0)
      herm_prefetch<UB, RB, N, AR>(in, (nu / upm) * (unsigned long long)D * D, (uint32_t)(nu % upm) << KH, t);
  };
  if (xb == 0) {
#pragma unroll 1
    for (uint32_t q = 0; q < (1u << (KH - KR)); ++q) {
      run_unit<UB, RB, N, AR, false, decltype(prefetch_ahead), MirrorUpperEpi>(in, out, base, q << KR, 0, xaddr,
                                                                               smax, t, prefetch_ahead);
      __syncthreads();
    }
  } else {
    run_unit_herm<UB, RB, N, AR>(in, out, base, xb, xaddr, smax, t, prefetch_ahead);
  }
}

template <int N, class AR>
cudaError_t launch_herm(const void* in, long long count, void* out, cudaStream_t st) {
  constexpr size_t smem = Unit<13, 4>::kSmem;
  constexpr int KH = 13 - (N - 1);
  auto kern = xordiag_herm_kernel<N, AR>;
  static bool ready = false;
  if (!ready) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ready = true;
  }
  const unsigned long long units = (unsigned long long)count * ((1ull << N) >> KH);
  if (units > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
  kern<<<(unsigned)units, Unit<13, 4>::kThreads, smem, st>>>(in, out, units, (unsigned long long)xk::device_sms());
  return cudaGetLastError();
}

template <class AR>
cudaError_t dispatch_herm(int N, const void* in, long long count, void* out, cudaStream_t st) {
  switch (N) {
    case 7: return launch_herm<7, AR>(in, count, out, st);
    case 8: return launch_herm<8, AR>(in, count, out, st);
    case 9: return launch_herm<9, AR>(in, count, out, st);
    case 10: return launch_herm<10, AR>(in, count, out, st);
    case 11: return launch_herm<11, AR>(in, count, out, st);
    case 12: return launch_herm<12, AR>(in, count, out, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace xh
}  // namespace pauli

// compose_batched.cuh -- one launch that composes a batch of coefficient vectors of uneven N,
// G_b = 2^scale_exp sum_n c_b[n] P_n (Eq. (1)), instantiated per dtype by compose_batched_*.cu.
//
// Work items: for N >= 6 one XOR-diagonal unit of 4096 elements (the composition unit of the
// single-matrix kernel: 2^(12-N) consecutive XY-masks x, all 2^N values of z gathered from c,
// the phase (-i)^popc(x&z), the transform over z -> r, and the store of G[r, r ^ x]); a smaller
// matrix is one item, composed whole in shared memory. The matrix table (largest N first, each
// entry with the index of its first item) is a kernel parameter, and CTAs take the items in a
// fixed stride (item i on CTA i mod gridDim): no device state, so a launch allocates nothing,
// needs no reset and can be captured in a graph with its own table.
#pragma once
#include "plan_internal.h"
#include "xordiag_impl.cuh"

namespace pauli {
namespace cb {
using namespace xd;

constexpr int kUB = 12;  // log2 elements per unit: 256 threads x 16, two CTAs per SM
constexpr int kMaxTable = 1024;
constexpr int kMaxN = 11;  // a unit holds at least two XY-masks

struct ComposeTable {
  PlanMat mats[kMaxTable];  // in = c, out = G
};
static_assert(sizeof(ComposeTable) + 32 <= 32764, "the table fits the kernel parameter limit");

// Whole N-qubit composition (N < 6) in one CTA: element u = x | (z << N) holds
// c(x, z) (-i)^popc(x&z) at a per-class fixed-point scale; N butterfly stages over the z bits
// give e_x[r] = G[r, r ^ x] at u = x | (r << N).
template <int N, class AR>
__device__ void run_small_compose(const void* __restrict__ in, void* __restrict__ out, int scale_exp, uint32_t xaddr,
                                  uint32_t* smax, uint32_t t, uint32_t T) {
  constexpr uint32_t D = 1u << N, E = D * D;
  constexpr int LPRE = N < 9 ? 9 - N : 0;
  if (AR::kScaled) {
    for (uint32_t i = t; i < D; i += T) smax[i] = 0u;
    __syncthreads();
  }
  for (uint32_t u = t; u < E; u += T) {
    const uint32_t x = u & (D - 1u), z = u >> N;
    const typename AR::Raw raw = AR::load(in, pauli_index(x, z));
    if (AR::kScaled) atomicMax(&smax[x], AR::exp_key(raw));
    sts128(xaddr + 16u * u, AR::raw_pack(raw));
  }
  __syncthreads();
  for (uint32_t u = t; u < E; u += T) {
    const uint32_t x = u & (D - 1u), z = u >> N;
    const typename AR::Conv cv = AR::make_conv(N, AR::kScaled ? smax[x] : 0u, scale_exp);
    const typename AR::Elem v =
        AR::template convert<LPRE>(AR::raw_unpack(lds128(xaddr + 16u * u)), cv, 3u * (uint32_t)__popc(x & z));
    sts128(xaddr + 16u * u, AR::pack(v));
  }
#pragma unroll
  for (int b = 0; b < N; ++b) {
    __syncthreads();
    for (uint32_t p = t; p < E / 2; p += T) {
      const uint32_t low = p & ((1u << (N + b)) - 1u);
      const uint32_t u0 = ((p >> (N + b)) << (N + b + 1)) | low, u1 = u0 | (1u << (N + b));
      typename AR::Elem a = AR::unpack(lds128(xaddr + 16u * u0)), e = AR::unpack(lds128(xaddr + 16u * u1));
      AR::bfly(a, e);
      sts128(xaddr + 16u * u0, AR::pack(a));
      sts128(xaddr + 16u * u1, AR::pack(e));
    }
  }
  __syncthreads();
  for (uint32_t u = t; u < E; u += T) {
    const uint32_t x = u & (D - 1u), r = u >> N;
    const typename AR::Conv cv = AR::make_conv(N, AR::kScaled ? smax[x] : 0u, scale_exp);
    AR::store(out, (unsigned long long)r * D + (r ^ x), AR::unpack(lds128(xaddr + 16u * u)), cv, 0u);
  }
  __syncthreads();  // the next item reuses the shared memory
}

// Matrix of item `cur`: the last table entry whose first item is <= cur (binary search).
__device__ __forceinline__ int table_find(const ComposeTable& tab, int batch, int cur) {
  int lo = 0, hi = batch - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab.mats[mid].first <= cur)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <class AR>
__global__ void __launch_bounds__((Unit<kUB, 4>::kThreads), (Unit<kUB, 4>::kMinBlocks))
    compose_batched_kernel(const __grid_constant__ ComposeTable tab, int batch, int n_items, int scale_exp) {
  extern __shared__ __align__(16) uint4 xbuf[];
  __shared__ uint32_t smax[64];
  const uint32_t t = threadIdx.x, T = blockDim.x;
  const uint32_t xaddr = (uint32_t)__cvta_generic_to_shared(xbuf);
  auto none = [] {};
  for (int cur = blockIdx.x; cur < n_items; cur += gridDim.x) {
    const int b = table_find(tab, batch, cur);
    const PlanMat& m = tab.mats[b];
    const uint32_t unit = (uint32_t)(cur - m.first);
#define CB_UNIT(NQ) \
  run_unit<kUB, 4, NQ, AR, true>(m.in, m.out, 0ull, unit << (kUB - NQ), scale_exp, xaddr, smax, t, none)
#define CB_SMALL(NQ) run_small_compose<NQ, AR>(m.in, m.out, scale_exp, xaddr, smax, t, T)
    switch (m.N) {
      case 1: CB_SMALL(1); break;
      case 2: CB_SMALL(2); break;
      case 3: CB_SMALL(3); break;
      case 4: CB_SMALL(4); break;
      case 5: CB_SMALL(5); break;
      case 6: CB_UNIT(6); break;
      case 7: CB_UNIT(7); break;
      case 8: CB_UNIT(8); break;
      case 9: CB_UNIT(9); break;
      case 10: CB_UNIT(10); break;
      case 11: CB_UNIT(11); break;
      default: break;
    }
#undef CB_UNIT
#undef CB_SMALL
    __syncthreads();  // shared memory and smax are reused by the next item
  }
}

// Items of an N-qubit matrix: 4096-element units from N = 6, else one.
__host__ __device__ inline unsigned items_of(int N) { return N >= 6 ? (unsigned)((1ull << (2 * N)) >> kUB) : 1u; }

template <class AR>
cudaError_t launch_t(const ComposeTable& tab, int batch, int n_items, int scale_exp, cudaStream_t s) {
  auto kern = compose_batched_kernel<AR>;
  constexpr size_t smem = Unit<kUB, 4>::kSmem;
  static int grid = 0;
  if (!grid) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Unit<kUB, 4>::kThreads, smem);
    if (e != cudaSuccess) return e;
    grid = sms * (per_sm > 0 ? per_sm : 1);
  }
  const int g = n_items < grid ? n_items : grid;
  kern<<<g, Unit<kUB, 4>::kThreads, smem, s>>>(tab, batch, n_items, scale_exp);
  return cudaGetLastError();
}

}  // namespace cb
}  // namespace pauli

// plan_kernels.cuh -- one persistent launch that decomposes a batch of matrices of uneven N.
//
// The plan's work list holds one item per work unit: for N at or above the unit size's
// threshold an item is one XOR-diagonal unit of the matrix (2^UB elements, the same unit the
// single-matrix kernel processes); a smaller matrix is one item, transformed whole in shared
// memory. Items are ordered by decreasing N (largest work first). Every CTA of the persistent
// grid takes items from a device counter, and fetches its next item early so that it can
// prefetch that item's rows into L2 while computing the current one. The counter and a
// status word live in a small control block that the plan resets before each launch.
#pragma once
#include <type_traits>

#include "kernels.h"
#include "plan_internal.h"
#include "xordiag_impl.cuh"

namespace pauli {
namespace pk {
using namespace xd;

static constexpr int kStallPolls = 1 << 17;  // ~0.1-1 s of polling before the wait gives up

// Whole N-qubit matrix (N <= 6) in one CTA: elements u = class | (row << N) in shared memory,
// per-class fixed-point scale, N butterfly stages in shared memory, phase and store.
// MIRROR: G is Hermitian and read from its upper triangle (an element below the diagonal is
// read as the conjugate of its mirror, the diagonal's imaginary parts are dropped).
template <int N, class AR, bool MIRROR = false>
__device__ void run_small(const void* __restrict__ in, void* __restrict__ out, uint32_t xaddr, uint32_t* smax,
                          uint32_t t, uint32_t T) {
  constexpr uint32_t D = 1u << N, E = D * D;
  constexpr int LPRE = N < 9 ? 9 - N : 0;
  if (AR::kScaled) {
    for (uint32_t i = t; i < D; i += T) smax[i] = 0u;
    __syncthreads();
  }
  for (uint32_t u = t; u < E; u += T) {
    const uint32_t c = u & (D - 1u), r = u >> N;
    typename AR::Raw raw;
    if constexpr (MIRROR) {
      const bool lower = c && ((r >> (31u - (uint32_t)__clz(c))) & 1u);
      if (lower) {
        raw = AR::conj(AR::load(in, (unsigned long long)(r ^ c) * D + r));
      } else {
        raw = AR::load(in, (unsigned long long)r * D + (r ^ c));
        if (c == 0u) raw = AR::real_part(raw);
      }
    } else {
      raw = AR::load(in, (unsigned long long)r * D + (r ^ c));
    }
    if (AR::kScaled) atomicMax(&smax[c], AR::exp_key(raw));
    sts128(xaddr + 16u * u, AR::raw_pack(raw));
  }
  __syncthreads();
  for (uint32_t u = t; u < E; u += T) {
    const typename AR::Conv cv = AR::make_conv(N, AR::kScaled ? smax[u & (D - 1u)] : 0u, -N);
    sts128(xaddr + 16u * u, AR::pack(AR::template convert<LPRE>(AR::raw_unpack(lds128(xaddr + 16u * u)), cv, 0u)));
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
    const uint32_t c = u & (D - 1u), z = u >> N;
    const typename AR::Conv cv = AR::make_conv(N, AR::kScaled ? smax[c] : 0u, -N);
    AR::store(out, pauli_index(c, z), AR::unpack(lds128(xaddr + 16u * u)), cv, (uint32_t)__popc(c & z));
  }
}

// L2 prefetch of every input row segment of item `it` (128-byte lines). HERM: the item's rows
// are those with bit h of the unit's classes clear (upper-triangle units, unit > 0).
__device__ __forceinline__ void prefetch_item(const PlanItem& it, const PlanMat& m, int UB, size_t esz, uint32_t t,
                                              uint32_t T, bool herm = false) {
  const uint32_t D = 1u << m.N;
  const int nmin = herm ? plan_min_herm_n(UB) : plan_min_unit_n(UB);
  const int small = m.N < nmin;
  const bool half = herm && !small && it.unit > 0;
  const int K = small ? m.N : UB - m.N + (half ? 1 : 0);
  const uint32_t seg = (1u << K) * (uint32_t)esz;  // bytes of the unit's classes in one row
  const uint32_t lines = seg > 128u ? seg / 128u : 1u;
  const uint32_t xb = small ? 0u : it.unit << (UB - m.N + (herm ? 1 : 0));
  const uint32_t lowm = half ? (1u << (31u - (uint32_t)__clz(xb))) - 1u : ~0u;
  const uint32_t rows = half ? D / 2 : D;
  const char* base = reinterpret_cast<const char*>(m.in);
  for (uint32_t i = t; i < rows * lines; i += T) {
    const uint32_t rr = i / lines, l = i % lines;
    const uint32_t r = half ? ((rr & lowm) | ((rr & ~lowm) << 1)) : rr;
    const unsigned long long col = (r ^ xb) & ~((1u << K) - 1u);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(base + ((unsigned long long)r * D + col) * esz + 128ull * l));
  }
}

// Item `cur` of a work list given only by the matrix table: mats[b].first is the index of
// matrix b's first item (table ordered as the work list), found by binary search.
__device__ __forceinline__ PlanItem item_from_table(int cur, const PlanMat* __restrict__ mats, int batch) {
  int lo = 0, hi = batch - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (mats[mid].first <= cur)
      lo = mid;
    else
      hi = mid - 1;
  }
  return PlanItem{(uint32_t)lo, (uint32_t)(cur - mats[lo].first)};
}

// One work unit of an N-qubit matrix (N >= the unit threshold). The Hermitian form is kept out
// of line: each N's body is compiled once, which keeps the build of the kernel short.
template <int UB, int N, class AR, bool HERM, class Prefetch>
__device__ __forceinline__ void plan_unit_inl(const PlanMat& m, uint32_t unit, uint32_t xaddr, uint32_t* smax, uint32_t t,
                                          Prefetch pf) {
  if constexpr (!HERM) {
    run_unit<UB, 4, N, AR, false>(m.in, m.out, 0ull, unit << (UB - N), 0, xaddr, smax, t, pf);
  } else if constexpr (2 * N <= UB) {
    // an upper-triangle unit would hold more classes than the matrix has: one full-row unit
    // holds the whole matrix (N = 6 with 4096-element units)
    run_unit<UB, 4, N, AR, false, Prefetch, MirrorUpperEpi>(m.in, m.out, 0ull, 0u, 0, xaddr, smax, t, pf);
  } else {
    constexpr int KH = UB - N + 1, KR = UB - N;
    if (unit == 0) {
#pragma unroll 1
      for (uint32_t q = 0; q < 2u; ++q) {
        run_unit<UB, 4, N, AR, false, Prefetch, MirrorUpperEpi>(m.in, m.out, 0ull, q << KR, 0, xaddr, smax, t, pf);
        __syncthreads();
      }
    } else {
      run_unit_herm<UB, 4, N, AR>(m.in, m.out, 0ull, unit << KH, xaddr, smax, t, pf);
    }
  }
}

template <int UB, int N, class AR, bool HERM, class Prefetch>
__device__ __noinline__ void plan_unit_call(const PlanMat& m, uint32_t unit, uint32_t xaddr, uint32_t* smax, uint32_t t,
                                            Prefetch pf) {
  plan_unit_inl<UB, N, AR, HERM>(m, unit, xaddr, smax, t, pf);
}
template <int UB, int N, class AR, bool HERM, class Prefetch>
__device__ __forceinline__ void plan_unit(const PlanMat& m, uint32_t unit, uint32_t xaddr, uint32_t* smax, uint32_t t,
                                          Prefetch pf) {
  if constexpr (HERM)
    plan_unit_call<UB, N, AR, HERM>(m, unit, xaddr, smax, t, pf);
  else
    plan_unit_inl<UB, N, AR, HERM>(m, unit, xaddr, smax, t, pf);
}

// HERM: every matrix is Hermitian and read from its upper triangle; AR stores real parts.
// Matrices from N = plan_min_herm_n(UB) on are cut into units of 2^(UB - N + 1) classes over
// half the rows (run_unit_herm); unit 0 (the diagonal and classes below 2^(UB - N + 1), of
// different top bits) runs as two full-row units with the lower triangle mirrored.
template <int UB, class AR, bool HERM = false>
__global__ void __launch_bounds__((Unit<UB, 4>::kThreads), (Unit<UB, 4>::kMinBlocks))
    plan_kernel(const PlanItem* __restrict__ items, int n_items, const PlanMat* __restrict__ mats, PlanCtrl* ctrl,
                int batch) {
  // The next item's rows are prefetched into L2 while this one computes; measured on GB300 the
  // prefetch pays for complex128 (general batch: 0.80 against 0.97 ms without) but not for
  // complex64 (0.79 against 0.78 ms; Hermitian batch 0.47 against 0.44 ms).
  constexpr bool kPrefetch = !std::is_same<AR, ArC64>::value && !std::is_same<AR, ReOut<ArC64>>::value;
  extern __shared__ __align__(16) uint4 xbuf[];
  __shared__ uint32_t smax[128];
  __shared__ int s_next;
  const uint32_t t = threadIdx.x, T = blockDim.x;
  const uint32_t xaddr = (uint32_t)__cvta_generic_to_shared(xbuf);
  constexpr size_t esz = sizeof(typename AR::Raw) == 16 ? 16 : 8;
  if (blockIdx.x == 0 && t == 0 && *(volatile int*)&ctrl->stall) {
    // Test hook: wait for a flag that nothing sets; give up after a bounded number of polls.
    int i = 0;
    for (; i < kStallPolls; ++i) {
      if (*(volatile int*)&ctrl->never) break;
      __nanosleep(2000);
    }
    if (i == kStallPolls) atomicExch(&ctrl->status, 8 /* PAULI_ERR_TIMEOUT */);
  }
  if (t == 0) s_next = atomicAdd(&ctrl->counter, 1);
  __syncthreads();
  int cur = s_next;
  while (cur < n_items) {
    __syncthreads();  // everyone has read s_next
    if (t == 0) s_next = atomicAdd(&ctrl->counter, 1);
    __syncthreads();
    const int nxt = s_next;
    const PlanItem it = items ? items[cur] : item_from_table(cur, mats, batch);
    const PlanMat m = mats[it.mat];
    auto pf = [&]() {
      if (kPrefetch && nxt < n_items) {
        const PlanItem in2 = items ? items[nxt] : item_from_table(nxt, mats, batch);
        prefetch_item(in2, mats[in2.mat], UB, esz, t, T, HERM);
      }
    };
#define PLAN_UNIT(NQ) plan_unit<UB, NQ, AR, HERM>(m, it.unit, xaddr, smax, t, pf)
#define PLAN_SMALL(NQ) \
  do {                 \
    pf();              \
    run_small<NQ, AR, HERM>(m.in, m.out, xaddr, smax, t, T); \
  } while (0)
    switch (m.N) {
      case 1: PLAN_SMALL(1); break;
      case 2: PLAN_SMALL(2); break;
      case 3: PLAN_SMALL(3); break;
      case 4: PLAN_SMALL(4); break;
      case 5: PLAN_SMALL(5); break;
      case 6:
        if constexpr (UB == 12) PLAN_UNIT(6); else PLAN_SMALL(6);
        break;
      case 7: PLAN_UNIT(7); break;
      case 8: PLAN_UNIT(8); break;
      case 9: PLAN_UNIT(9); break;
      case 10: PLAN_UNIT(10); break;
      default: break;
    }
#undef PLAN_UNIT
#undef PLAN_SMALL
    cur = nxt;
  }
}

template <int UB, class AR, bool HERM = false>
cudaError_t launch_plan_t(const PlanItem* items, int n_items, const PlanMat* mats, PlanCtrl* ctrl, int blocks_per_sm,
                          cudaStream_t s, int batch = 0) {
  auto kern = plan_kernel<UB, AR, HERM>;
  constexpr size_t smem = Unit<UB, 4>::kSmem;
  static int resident = 0;
  if (!resident) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, Unit<UB, 4>::kThreads, smem);
    if (e != cudaSuccess) return e;
    resident = n > 0 ? n : 1;
  }
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = blocks_per_sm > 0 && blocks_per_sm < resident ? blocks_per_sm : resident;
  kern<<<sms * per_sm, Unit<UB, 4>::kThreads, smem, s>>>(items, n_items, mats, ctrl, batch);
  return cudaGetLastError();
}

}  // namespace pk
}  // namespace pauli

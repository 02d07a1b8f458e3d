// tiled_impl.cuh -- kernel and launcher templates of the two-stage tiled decomposition
// (tiled.cu), instantiated per dtype and CTA shape by tiled_c128_u13.cu and its siblings.
//
// The decomposition for 12 <= N <= 14 in two stages through an L2-resident scratch ring.
//
// The single-pass kernels read, for one unit of XY-masks x, the element G[r, r^x] of every
// row r: 2^K consecutive masks give a 2^K-element run per row, and on-chip capacity forces K
// down as N grows (K = 1 from N = 12 on: 32 bytes of a 64-256 KiB row), which DRAM serves
// far below its copy bandwidth. This path splits the transform of Eq. (13) over the row
// index r = (R, i), R = r >> TB, i = r & (2^TB - 1), TB = UB - 6:
//
//  stage 1, per block of 64 XY-masks x = 64k + c and tile of 2^TB rows R: the elements
//    G[2^TB R + i, (2^TB R + i) ^ x] form a 2^TB x 64 block of G (each row one contiguous
//    run of 64 elements), and the tile's 64 classes get their TB low WHT stages (over i):
//        P[x][R][w] = sum_i (-1)^popc(i & w) e_x[2^TB R + i],   w < 2^TB,
//    in int64 fixed point with a per-(class, tile) scale (complex128), or as TwoSum pairs
//    (complex64), stored to a scratch slot together with the scale.
//  stage 2, per 8 classes and a group of w: the remaining N - TB stages over R,
//        W_x[(h << TB) | w] = sum_R (-1)^popc(R & h) P[x][R][w],
//    after re-scaling every tile to its class's largest scale (an exact arithmetic right
//    shift: a tile at a finer scale drops bits below the class quantum), then the phase
//    i^popc(x&z), the 2^-N scale and the store of c(x, z) in the paper's order (Eq. (2)).
//
// One persistent launch runs both stages from a single work counter, in the order
// S1(block 0), S1(1), S2(0), S1(2), S2(1), ...; the scratch is a ring of kTiledSlots slots of
// 64 x 2^N partials (16 MiB at N = 14), stored with an L2 evict-last policy so that it stays in
// L2, while G and c stream with evict-first. A stage-2 item waits until the 2^(N-TB) tiles of
// its block are complete, and a stage-1 item waits until the stage-2 items of the block that
// last used its slot have read it. Every item waited on was taken from the counter earlier by
// a CTA that is already running and finishes it without waiting on any later item, so all
// waits end; they are bounded anyway: after kPolls polls the waiting CTA records
// PAULI_ERR_TIMEOUT in the status word and carries on (its results are then not valid).
#pragma once
#include <cstddef>

#include "kernels.h"
#include "tiled.h"
#include "xordiag_impl.cuh"

namespace pauli {

// Scratch of at least `bytes` for launches on `st` (tiled.cu).
cudaError_t tiled_workspace(cudaStream_t st, size_t bytes, void** out);

namespace tiled {
namespace {
using namespace xd;

constexpr int kCB = 6;  // class bits per block
constexpr int kPolls = 1 << 22;
constexpr int kStatusTimeout = 8;  // PAULI_ERR_TIMEOUT

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// G is read once: no L1 allocation, evict-first in L2
template <class Raw>
__device__ __forceinline__ Raw ld_stream(const void* base, unsigned long long i, uint64_t pol);
template <>
__device__ __forceinline__ uint4 ld_stream<uint4>(const void* base, unsigned long long i, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(reinterpret_cast<const uint4*>(base) + i), "l"(pol));
  return v;
}
template <>
__device__ __forceinline__ float2 ld_stream<float2>(const void* base, unsigned long long i, uint64_t pol) {
  float2 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;"
               : "=f"(v.x), "=f"(v.y)
               : "l"(reinterpret_cast<const float2*>(base) + i), "l"(pol));
  return v;
}
// Scratch reads: written by other CTAs during this launch, so through L2 only (.cg), never the
// non-coherent path.
__device__ __forceinline__ uint4 ld_scratch(const uint4* a, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(a), "l"(pol)
               : "memory");
  return v;
}
__device__ __forceinline__ void st_hint(uint4* a, const uint4& v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(a), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 polls until *counter >= target (bounded), then the whole CTA proceeds.
__device__ __forceinline__ void wait_for(const int* counter, int target, int* status) {
  if (threadIdx.x == 0) {
    int i = 0;
    while (ld_acquire(counter) < target) {
      if (++i == kPolls) {
        atomicExch(status, kStatusTimeout);
        break;
      }
      __nanosleep(256);
    }
  }
  __syncthreads();
}
// All threads' prior accesses are ordered before the increment (barrier, then a fence by
// the thread that increments).
__device__ __forceinline__ void signal(int* counter) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1);
  }
}

// Scratch slot s: P[R][w][c] (16 bytes each: the int64 pair of complex128, or the two TwoSum
// float pairs of complex64), then E[R][c] (exponent key of each class in each tile).
struct Slot {
  uint4* P;
  uint32_t* E;
};
__host__ __device__ constexpr size_t slot_p_elems(int N) { return ((size_t)1 << N) << kCB; }
__host__ __device__ constexpr size_t slot_bytes(int N, int TB) {
  return slot_p_elems(N) * 16 + ((((size_t)1 << (N - TB)) << kCB) * 4 + 255) / 256 * 256;
}
__device__ __forceinline__ Slot slot_of(TiledCtrl* ws, int N, int TB, int s) {
  char* base = reinterpret_cast<char*>(ws) + kTiledCtrlBytes + (size_t)s * slot_bytes(N, TB);
  return Slot{reinterpret_cast<uint4*>(base), reinterpret_cast<uint32_t*>(base + slot_p_elems(N) * 16)};
}

// ---------------------------------------------------------------------------- stage 1 --
// Tile R of block k: rows [2^TB R, 2^TB (R+1)), classes [64k, 64k + 64).
template <int UB, int N, class AR>
__device__ __forceinline__ void stage1(const void* __restrict__ G, unsigned long long gbase, uint32_t k, uint32_t R,
                                       const Slot& sl, uint32_t xaddr, uint32_t* smax, uint64_t pol_in,
                                       uint64_t pol_keep) {
  constexpr int TB = UB - kCB;
  using LY = Layout<UB, TB, 4>;
  static_assert(LY::K == kCB, "tile = 64 classes x 2^TB rows");
  constexpr int E = LY::E, LAST = LY::NPH - 1;
  constexpr uint32_t D = 1u << N;
  const uint32_t t = threadIdx.x;
  const uint32_t c = t & 63u;
  const uint32_t row0 = R << TB;
  const uint32_t col0 = row0 ^ (k << kCB);        // (row0 + i) ^ (64k + c) = col0 ^ i ^ c
  const uint32_t it = LY::thread_u(0, t) >> kCB;  // thread part of the in-tile row
  typename AR::Raw raw[E];
  uint32_t emax = 0;
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const uint32_t i = it | (LY::reg_u(0, j) >> kCB);
    raw[j] = ld_stream<typename AR::Raw>(G, gbase + (unsigned long long)(row0 | i) * D + (col0 ^ i ^ c), pol_in);
    emax = max(emax, AR::exp_key(raw[j]));
  }
  uint32_t Ekey = 0;
  if constexpr (AR::kScaled) {
    if (t < 64) smax[t] = 0;
    __syncthreads();
    atomicMax(&smax[c], emax);  // lanes hold distinct classes: nothing to combine within a warp
    __syncthreads();
    Ekey = smax[c];
  }
  const typename AR::Conv cv = AR::make_conv(N, Ekey, 0);
  typename AR::Elem v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = AR::template convert<0>(raw[j], cv, 0u);
  local_wht<LY, AR>(v, xaddr, t);
  const uint32_t wt = LY::thread_u(LAST, t) >> kCB;
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const uint32_t w = wt | (LY::reg_u(LAST, j) >> kCB);
    st_hint(sl.P + ((size_t)(row0 | w) << kCB) + c, AR::pack(v[j]), pol_keep);
  }
  if constexpr (AR::kScaled) {
    if (t < 64) sl.E[(R << kCB) | t] = Ekey;
  }
}

// L2 prefetch of tile R of block k (the rows' 64-element runs).
template <int UB, int N, class AR>
__device__ __forceinline__ void stage1_prefetch(const void* G, unsigned long long gbase, uint32_t k, uint32_t R) {
  constexpr int TB = UB - kCB;
  constexpr uint32_t D = 1u << N;
  constexpr int kLineElems = 128 / (int)sizeof(typename AR::Raw);
  constexpr int kPerRow = 64 / kLineElems;
  constexpr int kLines = kPerRow << TB;  // 128-byte lines in the tile
  const char* base = reinterpret_cast<const char*>(G);
  for (int l = threadIdx.x; l < kLines; l += blockDim.x) {
    const uint32_t i = (uint32_t)l / kPerRow, part = (uint32_t)l % kPerRow;
    const uint32_t row = (R << TB) | i;
    const uint32_t col = ((row ^ (k << kCB)) & ~63u) + part * kLineElems;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(base + (gbase + (unsigned long long)row * D + col) *
                                                            sizeof(typename AR::Raw)));
  }
}

// ---------------------------------------------------------------------------- stage 2 --
// Item (o, q) of block k: classes 64k + 8o + [0, 8), w in [2^ZB q, 2^ZB (q+1)), all R.
template <int UB, int N, class AR>
__device__ __forceinline__ void stage2(void* __restrict__ out, unsigned long long obase, uint32_t k, uint32_t item,
                                       const Slot& sl, uint32_t xaddr, uint32_t* smax, uint32_t* sexp,
                                       int* s2_counter, uint64_t pol_out, uint64_t pol_drop) {
  constexpr int TB = UB - kCB;
  constexpr int L = N - TB;  // row-block bits transformed here
  using LY = Layout<UB, L, 4>;
  constexpr int K = LY::K, E = LY::E, LAST = LY::NPH - 1;
  constexpr int ZB = K - 3;  // log2 of the w values per item
  static_assert(K >= 3 && L >= 4, "stage-2 unit = 8 classes x 2^ZB w x 2^L row blocks");
  constexpr uint32_t NR = 1u << L;
  const uint32_t t = threadIdx.x;
  const uint32_t o = item & 7u, q = item >> 3;
  const uint32_t c8 = t & 7u;                         // class within the octet (lowest thread bits)
  const uint32_t w = (q << ZB) | ((t >> 3) & ((1u << ZB) - 1u));
  const uint32_t cls = (o << 3) | c8;                 // class within the block
  const uint32_t Rt = LY::thread_u(0, t) >> K;        // thread part of the row block
  typename AR::Elem v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const uint32_t Rb = Rt | (LY::reg_u(0, j) >> K);
    v[j] = AR::unpack(ld_scratch(sl.P + ((size_t)((Rb << TB) | w) << kCB) + cls, pol_drop));
  }
  if constexpr (AR::kScaled) {
    // exponent keys of the octet's classes in every tile -> shared memory, and their maximum
    if (t < 8) smax[t] = 0;
    uint32_t m = 0;
    for (uint32_t e = t; e < NR * 8; e += blockDim.x) {  // e & 7 == c8 (blockDim is a multiple of 8)
      const uint32_t key = __ldcg(sl.E + (((e >> 3) << kCB) | (o << 3) | (e & 7u)));
      sexp[e] = key;
      m = max(m, key);
    }
    m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, 8));
    m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, 16));
    __syncthreads();
    if ((t & 31u) < 8) atomicMax(&smax[c8], m);
  }
  signal(s2_counter);  // the slot has been read (the barrier inside also publishes smax, sexp)
  typename AR::Conv cv;
  if constexpr (AR::kScaled) {
    const uint32_t Emax = smax[c8];
    cv = AR::make_conv(N, Emax, -N);
    if (!cv.nan) {
      const int em = (int)(Emax >> 20);
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const uint32_t Rb = Rt | (LY::reg_u(0, j) >> K);
        // a tile at exponent et was converted at scale 2^(s + em - et): shift by em - et
        // (0 for the largest tiles; all-zero tiles have et = 0 and hold zeros)
        AR::align(v[j], min(em - (int)(sexp[(Rb << 3) | c8] >> 20), 63));
      }
    }
  } else {
    cv = AR::make_conv(N, 0u, -N);
  }
  local_wht<LY, AR>(v, xaddr, t);
  // c(x, z), x = 64k + cls, z = (h << TB) | w, h = ht | (register part)
  const uint32_t x = (k << kCB) | cls;
  const uint32_t ht = LY::thread_u(LAST, t) >> K;
  Addr<N, false> ao;
  ao.init(obase, x, (ht << TB) | w);
  BitSum<LY::regrow(LAST, 0) + TB, LY::regrow(LAST, 1) + TB, LY::regrow(LAST, 2) + TB, LY::regrow(LAST, 3) + TB> xo;
  xo.init(x);
  const uint32_t ko = (uint32_t)__popc(x & ((ht << TB) | w));
#pragma unroll
  for (int j = 0; j < E; ++j)
    AR::store_hint(out, ao.at((LY::reg_u(LAST, j) >> K) << TB), v[j], cv, ko + xo.at(j), pol_out);
}

template <int UB>
struct TiledShape {
  static constexpr int kThreads = 1 << (UB - 4);
  static constexpr int kMinBlocks = UB == 12 ? 2 : 1;
  static constexpr size_t kSmem = (size_t)16 << UB;
};

template <int UB, int N, class AR>
__global__ void __launch_bounds__(TiledShape<UB>::kThreads, TiledShape<UB>::kMinBlocks)
    tiled_kernel(const void* __restrict__ G, void* __restrict__ out, int count, TiledCtrl* ws) {
  constexpr int TB = UB - kCB;
  extern __shared__ __align__(16) uint4 xbuf[];
  __shared__ uint32_t smax[64];
  __shared__ uint32_t sexp[AR::kScaled ? (8 << (N - TB)) : 1];
  __shared__ int s_item;
  constexpr uint32_t D = 1u << N;
  constexpr int nb = 1 << (N - kCB);  // class blocks per matrix
  constexpr int n1 = 1 << (N - TB);   // stage-1 tiles per block
  constexpr int n2 = 1 << (N - TB);   // stage-2 items per block (8 octets x w groups)
  constexpr int group = n1 + n2;
  const int blocks = nb * count;
  const int n_items = (blocks + 1) * group;
  const uint32_t xaddr = (uint32_t)__cvta_generic_to_shared(xbuf);
  const uint64_t pol_keep = policy_evict_last(), pol_stream = policy_evict_first();
  for (;;) {
    __syncthreads();  // s_item and shared buffers are free
    if (threadIdx.x == 0) s_item = atomicAdd(&ws->counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= n_items) break;
    const int g = item / group, j = item % group;
    if (j < n1) {
      if (g >= blocks) continue;
      const int b = g, s = b % kTiledSlots, gen = b / kTiledSlots;
      const unsigned long long gbase = (unsigned long long)(b / nb) * D * D;
      // the tile one resident wave ahead, when that item is a stage-1 tile too
      const int nx = item + (int)gridDim.x, gn = nx / group, jn = nx % group;
      if (jn < n1 && gn < blocks)
        stage1_prefetch<UB, N, AR>(G, (unsigned long long)(gn / nb) * D * D, (uint32_t)(gn % nb), (uint32_t)jn);
      if (gen > 0) wait_for(&ws->s2_done[s], n2 * gen, &ws->status);
      stage1<UB, N, AR>(G, gbase, (uint32_t)(b % nb), (uint32_t)j, slot_of(ws, N, TB, s), xaddr, smax, pol_stream,
                        pol_keep);
      signal(&ws->s1_done[s]);
    } else {
      if (g == 0) continue;
      const int b = g - 1, s = b % kTiledSlots, gen = b / kTiledSlots;
      wait_for(&ws->s1_done[s], n1 * (gen + 1), &ws->status);
      stage2<UB, N, AR>(out, (unsigned long long)(b / nb) * D * D, (uint32_t)(b % nb), (uint32_t)(j - n1),
                        slot_of(ws, N, TB, s), xaddr, smax, sexp, &ws->s2_done[s], pol_stream, pol_stream);
    }
  }
}

template <int UB, int N, class AR>
cudaError_t launch_tiled_t(const void* G, int count, void* out, cudaStream_t st) {
  constexpr int TB = UB - kCB;
  const size_t bytes = kTiledCtrlBytes + (size_t)kTiledSlots * slot_bytes(N, TB);
  void* ws = nullptr;
  cudaError_t e = tiled_workspace(st, bytes, &ws);
  if (e != cudaSuccess) return e;
  auto kern = tiled_kernel<UB, N, AR>;
  static int grid = 0;  // one wave of resident CTAs
  if (!grid) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TiledShape<UB>::kSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TiledShape<UB>::kThreads, TiledShape<UB>::kSmem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    grid = sms * per_sm;
  }
  // clear the counters (not the status word, which the host reads and clears)
  e = cudaMemsetAsync(ws, 0, offsetof(TiledCtrl, status), st);
  if (e != cudaSuccess) return e;
  kern<<<grid, TiledShape<UB>::kThreads, TiledShape<UB>::kSmem, st>>>(G, out, count, reinterpret_cast<TiledCtrl*>(ws));
  return cudaGetLastError();
}

template <int UB, class AR>
cudaError_t launch_tiled_n(const void* G, int N, int count, void* out, cudaStream_t st) {
  switch (N) {
    case 12: return launch_tiled_t<UB, 12, AR>(G, count, out, st);
    case 13: return launch_tiled_t<UB, 13, AR>(G, count, out, st);
    case 14: return launch_tiled_t<UB, 14, AR>(G, count, out, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace
}  // namespace tiled
}  // namespace pauli

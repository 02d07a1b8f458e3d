// tiled_impl.cuh -- kernel and launcher templates of the two-stage tiled decomposition
// (host side in tiled.cu), instantiated per dtype and consumer shape by tiled_c128_r3.cu and
// its siblings.
//
// The decomposition for 12 <= N <= 14 in two stages through an L2-resident scratch ring.
//
// The single-pass kernels read, for one unit of XY-masks x, the element G[r, r^x] of every
// row r: 2^K consecutive masks give a 2^K-element run per row, and on-chip capacity forces K
// down as N grows (K = 1 from N = 12 on: 32 bytes of a 64-256 KiB row), which DRAM serves
// far below its copy bandwidth. This path splits the transform of Eq. (13) over the row
// index r = (R, i), R = r >> 6, i = r & 63:
//
//  stage 1, per block of 64 XY-masks x = 64k + c and tile of 64 rows R: the elements
//    G[64R + i, (64R + i) ^ x] are the 64 x 64 submatrix of G at rows 64R.., columns
//    (64R ^ 64k).. (element (i, c) at column offset i ^ c), whose rows are contiguous 64-element
//    runs; the tile's 64 classes get their 6 low WHT stages (over i):
//        P[x][R][w] = sum_i (-1)^popc(i & w) e_x[64R + i],   w < 64,
//    in int64 fixed point with a per-(class, tile) scale (complex128), or as TwoSum pairs
//    (complex64), stored to a scratch slot together with the scale.
//  stage 2, per 8 classes (an octet) and a group of 2^ZB values of w: the remaining L = N - 6
//    stages over R,
//        W_x[(h << 6) | w] = sum_R (-1)^popc(R & h) P[x][R][w],
//    after re-scaling every tile to its class's largest scale (an arithmetic right shift: a
//    tile at a finer scale drops bits below the class quantum), then the phase i^popc(x&z),
//    the 2^-N scale and the store of c(x, z) in the paper's order (Eq. (2)).
//
// The scratch is laid out so that each stage-2 item reads one contiguous 64 KiB chunk:
// P[o][q][R][wl][c8] (octet o, w = (q << ZB) | wl, class 8o + c8), 16 bytes per entry,
// then E[o][R][c8] (exponent key of each class in each tile). A ring of kTiledSlots slots
// holds 64 x 2^N partials each (16 MiB at N = 14); it is written with an L2 evict-last policy
// and stays in L2 while G and c stream through with evict-first.
//
// Launch: one persistent CTA per SM, warp-specialised. A producer warp takes work items from
// a global counter in the order S1(block 0), S1(1), S2(0), S1(2), S2(1), ..., waits for the
// item's dependencies (a stage-2 item needs the 2^L tiles of its block; a stage-1 item needs
// the stage-2 items of the block that last used its slot to have copied their data out), and
// fills a 3-deep ring of shared-memory buffers with cp.async.bulk copies (64 row runs of 1 KiB
// for a tile of complex128 G, one chunk for a stage-2 item) that complete on an mbarrier. The
// consumer warps (512 threads x 8 elements or 256 x 16) take the buffers in order, compute,
// store, publish completion with a release reduction and hand the buffer back. Loads for the
// next two items are thus in flight while one is computed.
//
// Every item waited on was taken from the counter earlier by a CTA that processes its items in
// the order it took them, so every wait ends. Each wait is bounded nevertheless: after
// kPolls polls the waiting thread records PAULI_ERR_TIMEOUT in the status word, the CTA stops
// taking work, waits (bounded) for its copies in flight and exits; the results are then invalid.
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

constexpr int kCB = 6;             // class bits per block
constexpr int kUB = 12;            // log2 elements per item
constexpr int kTB = kUB - kCB;     // log2 rows per stage-1 tile
constexpr int kBufs = 3;           // shared-memory ring depth
constexpr int kPolls = 1 << 24;    // bound of every wait loop (each poll sleeps or blocks briefly)
constexpr int kStatusTimeout = 8;  // PAULI_ERR_TIMEOUT

template <int N>
struct Geo {
  static constexpr int L = N - kTB;        // stage-2 bits (row blocks)
  static constexpr int K2 = kUB - L;       // stage-2 class bits: 3 (octet) + ZB (w)
  static constexpr int ZB = K2 - 3;
  static constexpr int NR = 1 << L;        // tiles per block
  static constexpr int NQ = 1 << (kTB - ZB);  // w groups per octet
  static constexpr int n1 = NR;            // stage-1 items per block
  static constexpr int n2 = 8 * NQ;        // stage-2 items per block
  static constexpr size_t kChunk = (size_t)16 << kUB;          // bytes per item (64 KiB)
  static constexpr size_t kEOct = (size_t)NR * 8 * 4;          // E bytes per octet
  static constexpr size_t kBuf = kChunk + kEOct + 128;         // buffer: data, E, class maxima
  static constexpr size_t kSlotP = (size_t)16 << (N + kCB);
  static constexpr size_t kSlot = kSlotP + (size_t)NR * 64 * 4;
  static constexpr size_t kWorkspace = kTiledCtrlBytes + kTiledSlots * kSlot;
  static_assert(ZB >= 0 && L >= 4, "12 <= N <= 15");
  static_assert(n1 == n2, "both stages have 2^L items per block");
};

// ------------------------------------------------------------------- PTX helpers --
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
__device__ __forceinline__ void st_hint(void* a, const uint4& v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(a), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_max(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.max.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared bulk copy completing on mbarrier `bar` (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(pol)
      : "memory");
}

// Shared state of one CTA.
struct Shared {
  uint64_t full[kBufs];   // buffer filled (producer arrival + copied bytes)
  uint64_t empty[kBufs];  // buffer released by the consumers
  int item[kBufs];        // work item in the buffer, -1 = no more work
  int abort;              // a wait of the producer gave up: stop
  int ok;                 // consumers: the next buffer arrived (broadcast by consumer 0)
  int consumed;           // buffer uses completed by the consumers
  int issued;             // buffer uses whose copies the producer has issued
  uint32_t smax[64];      // stage 1: (use + 1) << 11 | largest exponent of each class
};

// Bounded wait on an mbarrier phase; false (status recorded) when it gave up.
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity, int* status) {
  for (int i = 0; i < kPolls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(status, kStatusTimeout);
  return false;
}
// Bounded wait until *counter >= target (one thread); false (status recorded) when it gave up.
__device__ __forceinline__ bool wait_count(const int* counter, int target, int* status) {
  for (int i = 0; i < kPolls; ++i) {
    if (ld_acquire(counter) >= target) return true;
    __nanosleep(128);
  }
  atomicExch(status, kStatusTimeout);
  return false;
}

// Work item -> (stage, block, index within the block); false for the padding items of the
// order (stage 1 past the last block, stage 2 before the first).
template <int N>
struct Item {
  bool s1;
  int b, j;
  __device__ __forceinline__ bool decode(int item, int blocks) {
    constexpr int group = Geo<N>::n1 + Geo<N>::n2;
    const int g = item / group, r = item % group;
    s1 = r < Geo<N>::n1;
    b = s1 ? g : g - 1;
    j = s1 ? r : r - Geo<N>::n1;
    return s1 ? g < blocks : g > 0;
  }
};

__device__ __forceinline__ char* slot_base(TiledCtrl* ws, size_t slot_bytes, int s) {
  return reinterpret_cast<char*>(ws) + kTiledCtrlBytes + (size_t)s * slot_bytes;
}

// ---------------------------------------------------------------------- producer --
template <int N, class AR>
__device__ void producer(const void* __restrict__ G, int count, TiledCtrl* ws, Shared& sh, uint32_t buf0) {
  using GE = Geo<N>;
  constexpr uint32_t D = 1u << N;
  constexpr int nb = 1 << (N - kCB);
  constexpr uint32_t kRowBytes = 64u * sizeof(typename AR::Raw);
  const int lane = threadIdx.x & 31;
  const int blocks = nb * count;
  const int n_items = (blocks + 1) * (GE::n1 + GE::n2);
  const uint64_t pol_first = policy_evict_first();
  int next = 0;
  if (lane == 0) next = atomicAdd(&ws->counter, 1);
  next = __shfl_sync(0xFFFFFFFFu, next, 0);
  int use = 0;
  for (;;) {
    const int item = next;
    const bool done = item >= n_items;
    Item<N> it;
    bool real = false;
    if (!done) {
      if (lane == 0) next = atomicAdd(&ws->counter, 1);  // latency overlaps the rest of this item
      next = __shfl_sync(0xFFFFFFFFu, next, 0);
      real = it.decode(item, blocks);
      if (!real) continue;
    }
    const int buf = use % kBufs;
    const uint32_t full = (uint32_t)__cvta_generic_to_shared(&sh.full[buf]);
    const uint32_t empty = (uint32_t)__cvta_generic_to_shared(&sh.empty[buf]);
    bool ok = true;
    if (lane == 0 && use >= kBufs) ok = wait_phase(empty, ((use / kBufs) - 1) & 1, &ws->status);
    ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
    if (!ok) {  // the consumers never released the buffer: they time out on their own wait
      if (lane == 0) sh.abort = 1;
      break;
    }
    const int s = done ? 0 : it.b % kTiledSlots, gen = done ? 0 : it.b / kTiledSlots;
    if (lane == 0 && !done) {
      // dependencies: the slot must be free (stage 1) or complete (stage 2)
      if (it.s1) {
        if (gen > 0) ok = wait_count(&ws->s2_done[s], GE::n2 * gen, &ws->status);
      } else {
        ok = wait_count(&ws->s1_done[s], GE::n1 * (gen + 1), &ws->status);
        // the chunk was written through the generic proxy; the copy reads it through the async one
        asm volatile("fence.proxy.async.global;" ::: "memory");
      }
    }
    ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
    if (done || !ok) {  // no more work (or a dependency never came): tell the consumers
      if (lane == 0) {
        if (!ok) sh.abort = 1;
        sh.item[buf] = -1;
        mbar_arrive(full);
      }
      break;
    }
    const uint32_t dst = buf0 + (uint32_t)(buf * GE::kBuf);
    if (lane == 0) {
      sh.item[buf] = item;
      const uint32_t bytes = it.s1 ? kRowBytes * 64u : (uint32_t)(GE::kChunk + GE::kEOct + 32);
      mbar_arrive_tx(full, bytes);
    }
    __syncwarp();
    if (it.s1) {
      const uint32_t k = (uint32_t)(it.b % nb), R = (uint32_t)it.j;
      const uint32_t row0 = R << kTB, colb = (row0 ^ (k << kCB)) & ~63u;
      const char* base = reinterpret_cast<const char*>(G) +
                         (size_t)(it.b / nb) * D * D * sizeof(typename AR::Raw);
      for (int r = lane; r < 64; r += 32)
        bulk_g2s(dst + (uint32_t)r * kRowBytes,
                 base + ((size_t)(row0 + r) * D + colb) * sizeof(typename AR::Raw), kRowBytes, full, pol_first);
    } else if (lane == 0) {
      const uint32_t o = (uint32_t)it.j & 7u, q = (uint32_t)it.j >> 3;
      char* sb = slot_base(ws, GE::kSlot, s);
      bulk_g2s(dst, sb + (size_t)(o * GE::NQ + q) * GE::kChunk, (uint32_t)GE::kChunk, full, pol_first);
      bulk_g2s(dst + (uint32_t)GE::kChunk, sb + GE::kSlotP + (size_t)o * GE::kEOct, (uint32_t)GE::kEOct, full,
               pol_first);
      bulk_g2s(dst + (uint32_t)(GE::kChunk + GE::kEOct), &ws->emax[s][o * 8], 32u, full, pol_first);
    }
    ++use;
    if (lane == 0) sh.issued = use;
  }
}

// ---------------------------------------------------------------------- stage 1 --
// Tile R of block k from the buffer: element (i, c) at 16-byte slot (i << 6) | (i ^ c).
template <int N, int RB, class AR, int CT>
__device__ __forceinline__ void stage1(uint32_t tile, char* slot, TiledCtrl* ws, int s, int gen, uint32_t R,
                                       Shared& sh, uint32_t tag, uint64_t pol_keep) {
  using GE = Geo<N>;
  using LY = Layout<kUB, kTB, RB>;
  using SY = NamedSync<1, CT>;
  static_assert(LY::K == kCB, "tile = 64 classes x 64 rows");
  constexpr int E = LY::E, LAST = LY::NPH - 1;
  constexpr uint32_t kEs = sizeof(typename AR::Raw);
  const uint32_t t = threadIdx.x;
  const uint32_t c = t & 63u;
  const uint32_t it = LY::thread_u(0, t) >> kCB;
  typename AR::Raw raw[E];
  uint32_t emax = 0;
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const uint32_t i = it | (LY::reg_u(0, j) >> kCB);
    const uint32_t a = tile + ((i << 6) | (i ^ c)) * kEs;
    if constexpr (kEs == 16) {
      raw[j] = AR::raw_unpack(lds128(a));
    } else {
      uint32_t x, y;
      asm volatile("ld.shared.v2.u32 {%0,%1}, [%2];" : "=r"(x), "=r"(y) : "r"(a) : "memory");
      raw[j] = AR::raw_unpack(make_uint4(x, y, 0u, 0u));
    }
    emax = max(emax, AR::exp_key(raw[j]));
  }
  uint32_t Ekey = 0;
  if constexpr (AR::kScaled) {
    atomicMax(&sh.smax[c], (tag << 11) | (emax >> 20));  // older tags are smaller: no reset needed
    SY::sync();
    Ekey = (sh.smax[c] & 0x7FFu) << 20;
  }
  const typename AR::Conv cv = AR::make_conv(N, Ekey, 0);
  typename AR::Elem v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = AR::template convert<0>(raw[j], cv, 0u);
  local_wht<LY, AR, 0, SY>(v, tile, t);  // the first exchange barrier also ends the tile reads
  // P[o][q][R][wl][c8]: o = c >> 3, c8 = c & 7, w = (q << ZB) | wl
  const uint32_t wt = LY::thread_u(LAST, t) >> kCB;
  uint4* P = reinterpret_cast<uint4*>(slot);
  const size_t cbase = (size_t)(c >> 3) * GE::NQ * (GE::kChunk / 16) + (c & 7u);
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const uint32_t w = wt | (LY::reg_u(LAST, j) >> kCB);
    const uint32_t q = w >> GE::ZB, wl = w & ((1u << GE::ZB) - 1u);
    st_hint(P + cbase + (size_t)q * (GE::kChunk / 16) + (((R << GE::ZB) | wl) << 3), AR::pack(v[j]), pol_keep);
  }
  if (t < 64) {
    uint32_t* Ep = reinterpret_cast<uint32_t*>(slot + GE::kSlotP);
    Ep[((t >> 3) * GE::NR + R) * 8 + (t & 7u)] = Ekey;
    if constexpr (AR::kScaled) red_max(&ws->emax[s][t], ((uint32_t)(gen + 1) << 11) | (Ekey >> 20));
  }
}

// ---------------------------------------------------------------------- stage 2 --
// Item j = (o, q) of block k: the chunk holds entry (R, wl, c8) at 16-byte slot
// (R << K2) | (wl << 3) | c8 -- the unit's own element order -- then E[R][c8], then the
// eight tagged class maxima.
template <int N, int RB, class AR, int CT>
__device__ __forceinline__ void stage2(uint32_t chunk, const char* chunk_gen, void* __restrict__ out,
                                       unsigned long long obase, uint32_t k, uint32_t item, uint64_t pol_out) {
  using GE = Geo<N>;
  using LY = Layout<kUB, GE::L, RB>;
  using SY = NamedSync<1, CT>;
  constexpr int K = LY::K, E = LY::E, LAST = LY::NPH - 1, ZB = GE::ZB;
  static_assert(K == GE::K2, "stage-2 unit = 8 classes x 2^ZB w x 2^L row blocks");
  const uint32_t t = threadIdx.x;
  const uint32_t o = item & 7u, q = item >> 3;
  const uint32_t c8 = t & 7u;
  const uint32_t w = (q << ZB) | ((t >> 3) & ((1u << ZB) - 1u));
  const uint32_t x = (k << kCB) | (o << 3) | c8;
  const uint32_t u0 = LY::thread_u(0, t);
  typename AR::Elem v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = AR::unpack(lds128(chunk + 16u * (u0 | LY::reg_u(0, j))));
  typename AR::Conv cv;
  if constexpr (AR::kScaled) {
    const uint32_t* Es = reinterpret_cast<const uint32_t*>(chunk_gen + GE::kChunk);
    const int em = (int)(Es[GE::NR * 8 + c8] & 0x7FFu);
    cv = AR::make_conv(N, (uint32_t)em << 20, -N);
    if (!cv.nan) {
      const uint32_t Rt = u0 >> K;
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const uint32_t Rb = Rt | (LY::reg_u(0, j) >> K);
        // tile at exponent et was converted at scale 2^(s + em - et): shift right by em - et
        // (all-zero tiles have et = 0 and hold zeros)
        AR::align(v[j], min(em - (int)(Es[(Rb << 3) | c8] >> 20), 63));
      }
    }
  } else {
    cv = AR::make_conv(N, 0u, -N);
  }
  local_wht<LY, AR, 0, SY>(v, chunk, t);  // the first exchange barrier also ends the chunk reads
  // c(x, z), z = (h << 6) | w, h = ht | (register part)
  const uint32_t ht = LY::thread_u(LAST, t) >> K;
  Addr<N, false> ao;
  ao.init(obase, x, (ht << kTB) | w);
  constexpr int p0 = LY::regrow(LAST, 0) < 0 ? -1 : LY::regrow(LAST, 0) + kTB;
  constexpr int p1 = LY::regrow(LAST, 1) < 0 ? -1 : LY::regrow(LAST, 1) + kTB;
  constexpr int p2 = LY::regrow(LAST, 2) < 0 ? -1 : LY::regrow(LAST, 2) + kTB;
  constexpr int p3 = LY::regrow(LAST, 3) < 0 ? -1 : LY::regrow(LAST, 3) + kTB;
  BitSum<p0, p1, p2, p3> xo;
  xo.init(x);
  const uint32_t ko = (uint32_t)__popc(x & ((ht << kTB) | w));
#pragma unroll
  for (int j = 0; j < E; ++j)
    AR::store_hint(out, ao.at((LY::reg_u(LAST, j) >> K) << kTB), v[j], cv, ko + xo.at(j), pol_out);
}

// ---------------------------------------------------------------------- consumers --
template <int N, int RB, class AR, int CT>
__device__ void consumer(void* __restrict__ out, int count, TiledCtrl* ws, Shared& sh, char* bufs, uint32_t buf0) {
  using GE = Geo<N>;
  using SY = NamedSync<1, CT>;
  constexpr uint32_t D = 1u << N;
  constexpr int nb = 1 << (N - kCB);
  const uint32_t t = threadIdx.x;
  const int blocks = nb * count;
  const uint64_t pol_keep = policy_evict_last(), pol_first = policy_evict_first();
  for (int use = 0;; ++use) {
    const int buf = use % kBufs;
    const uint32_t full = (uint32_t)__cvta_generic_to_shared(&sh.full[buf]);
    const uint32_t parity = (use / kBufs) & 1;
    // consumer 0 waits (bounded) and broadcasts, so that all consumers leave together
    if (t == 0) sh.ok = wait_phase(full, parity, &ws->status);
    SY::sync();
    if (!sh.ok) break;
    for (int i = 0; i < kPolls && !mbar_try_wait(full, parity); ++i) {  // completes at once: acquires the data
    }
    const int item = sh.item[buf];
    if (item < 0) break;
    Item<N> it;
    it.decode(item, blocks);
    const int s = it.b % kTiledSlots, gen = it.b / kTiledSlots;
    const uint32_t addr = buf0 + (uint32_t)(buf * GE::kBuf);
    if (it.s1) {
      stage1<N, RB, AR, CT>(addr, slot_base(ws, GE::kSlot, s), ws, s, gen, (uint32_t)it.j, sh, (uint32_t)use + 1u,
                            pol_keep);
    } else {
      if (t == 0) red_release_add(&ws->s2_done[s], 1);  // the slot's data is in shared memory now
      stage2<N, RB, AR, CT>(addr, bufs + (size_t)buf * GE::kBuf, out, (unsigned long long)(it.b / nb) * D * D,
                            (uint32_t)(it.b % nb), (uint32_t)it.j, pol_first);
    }
    SY::sync();  // every consumer is done with the buffer and has issued its stores
    if (t == 0) {
      if (it.s1) red_release_add(&ws->s1_done[s], 1);
      sh.consumed = use + 1;
      // the buffer was read and written through the generic proxy; the next copy writes it
      // through the async one
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive((uint32_t)__cvta_generic_to_shared(&sh.empty[buf]));
    }
  }
}

template <int RB>
struct TiledShape {
  static constexpr int kConsumers = 1 << (kUB - RB);
  static constexpr int kThreads = kConsumers + 32;
};

template <int N, int RB, class AR>
__global__ void __launch_bounds__(TiledShape<RB>::kThreads, 1)
    tiled_kernel(const void* __restrict__ G, void* __restrict__ out, int count, TiledCtrl* ws) {
  constexpr int CT = TiledShape<RB>::kConsumers;
  extern __shared__ __align__(1024) char bufs[];
  __shared__ Shared sh;
  const uint32_t t = threadIdx.x;
  const uint32_t buf0 = (uint32_t)__cvta_generic_to_shared(bufs);
  if (t == 0) {
    for (int b = 0; b < kBufs; ++b) {
      mbar_init((uint32_t)__cvta_generic_to_shared(&sh.full[b]), 1);
      mbar_init((uint32_t)__cvta_generic_to_shared(&sh.empty[b]), 1);
    }
    sh.abort = 0;
    sh.consumed = 0;
    sh.issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (t < 64) sh.smax[t] = 0;
  __syncthreads();
  if (t >= (uint32_t)CT) {
    producer<N, AR>(G, count, ws, sh, buf0);
  } else {
    consumer<N, RB, AR, CT>(out, count, ws, sh, bufs, buf0);
  }
  __syncthreads();
  // after a wait gave up: wait (bounded) for copies still landing in buffers nobody consumed
  if (t == (uint32_t)CT && sh.issued > sh.consumed) {
    for (int use = sh.consumed; use < sh.issued; ++use) {
      const uint32_t full = (uint32_t)__cvta_generic_to_shared(&sh.full[use % kBufs]);
      for (int i = 0; i < kPolls && !mbar_try_wait(full, (use / kBufs) & 1); ++i) {
      }
    }
  }
}

template <int N, int RB, class AR>
cudaError_t launch_tiled_t(const void* G, int count, void* out, cudaStream_t st) {
  using GE = Geo<N>;
  void* ws = nullptr;
  cudaError_t e = tiled_workspace(st, GE::kWorkspace, &ws);
  if (e != cudaSuccess) return e;
  auto kern = tiled_kernel<N, RB, AR>;
  constexpr size_t smem = kBufs * GE::kBuf;
  static int grid = 0;  // one CTA per SM
  if (!grid) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TiledShape<RB>::kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    grid = sms;
  }
  // clear the counters and class maxima, not the status word
  e = cudaMemsetAsync(reinterpret_cast<char*>(ws) + offsetof(TiledCtrl, counter), 0,
                      sizeof(TiledCtrl) - offsetof(TiledCtrl, counter), st);
  if (e != cudaSuccess) return e;
  kern<<<grid, TiledShape<RB>::kThreads, smem, st>>>(G, out, count, reinterpret_cast<TiledCtrl*>(ws));
  return cudaGetLastError();
}

template <int RB, class AR>
cudaError_t launch_tiled_n(const void* G, int N, int count, void* out, cudaStream_t st) {
  switch (N) {
    case 12: return launch_tiled_t<12, RB, AR>(G, count, out, st);
    case 13: return launch_tiled_t<13, RB, AR>(G, count, out, st);
    case 14: return launch_tiled_t<14, RB, AR>(G, count, out, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace
}  // namespace tiled
}  // namespace pauli

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
// then E[o][R][c8] (exponent key of each class in each tile). A ring of Geo<N>::NS slots
// holds 64 x 2^N partials each (16 MiB at N = 14; 3 to 6 slots by N); it is written with an L2
// evict-last policy and stays in L2 while G and c stream through with evict-first.
//
// Launch: one persistent CTA per SM, warp-specialised.
//  - a producer warp takes work items from a global counter in the order S1(block 0), ...,
//    S1(LAG), S2(0), S1(LAG + 1), S2(1), ..., waits for the item's dependencies (a stage-2 item
//    needs the 2^L tiles of its block; a stage-1 item needs the stage-2 items of the block that
//    last used its slot to have copied their data out), and fills a 3-deep ring of
//    shared-memory buffers: one 2D TMA tensor load per stage-1 tile (64 rows of 64 elements),
//    one bulk copy per stage-2 chunk, completing on the buffer's mbarrier;
//  - the consumers take the buffers in order: one group of 512 threads x 8 elements, or two
//    groups of 256 threads x 16 elements that take alternate buffers (so that one group's
//    arithmetic overlaps the other's shared-memory phases); each warp hands the buffer back
//    (mbarrier) as soon as it is done with it;
//  - a release warp publishes each finished stage-1 tile to the other SMs (a release reduction
//    on the slot's counter, which waits for the tile's stores to reach L2) off the consumers'
//    critical path.
//
// Every item waited on was taken from the counter earlier (the producer takes items in
// order), and an item whose copies a CTA has issued is finished by its consumers without
// waiting on any other item, so every wait ends. Each wait is bounded nevertheless: after
// kPolls polls the waiting thread records PAULI_ERR_TIMEOUT in the status word, the CTA stops
// taking work, waits (bounded) for its copies in flight and exits; the results are then invalid.
#pragma once
#include <cuda.h>

#include <cstddef>

#include "kernels.h"
#include "tiled.h"
#include "xordiag_impl.cuh"

namespace pauli {

// Scratch of at least `bytes` for launches on `st` (tiled.cu).
cudaError_t tiled_workspace(cudaStream_t st, size_t bytes, void** out);
// 2D tensor map of `count` stacked D x D matrices with `elem` bytes per element, box of
// 64 rows x 64 elements (tiled.cu).
cudaError_t tiled_tensor_map(CUtensorMap* map, const void* G, int N, int count, int elem);

namespace tiled {
namespace {
using namespace xd;

constexpr int kCB = 6;             // class bits per block
constexpr int kUB = 12;            // log2 elements per item
constexpr int kTB = kUB - kCB;     // log2 rows per stage-1 tile
constexpr int kBufs = 3;           // shared-memory ring depth
constexpr int kPolls = 1 << 24;    // bound of every wait loop (each poll sleeps or blocks briefly)
constexpr int kStatusTimeout = 8;  // PAULI_ERR_TIMEOUT
constexpr int kStallPolls = 1 << 15;  // the test hook's wait: well under a second

template <int N>
struct Geo {
  static constexpr int L = N - kTB;           // stage-2 bits (row blocks)
  static constexpr int K2 = kUB - L;          // stage-2 class bits: 3 (octet) + ZB (w)
  static constexpr int ZB = K2 - 3;
  static constexpr int NR = 1 << L;           // tiles per block
  static constexpr int NQ = 1 << (kTB - ZB);  // w groups per octet
  static constexpr int n1 = NR;               // stage-1 items per block
  static constexpr int n2 = 8 * NQ;           // stage-2 items per block
  static constexpr size_t kChunk = (size_t)16 << kUB;   // bytes per item (64 KiB)
  static constexpr size_t kEOct = (size_t)NR * 8 * 4;   // E bytes per octet
  static constexpr size_t kBuf = kChunk + kEOct + 128;  // buffer: data, E, class maxima
  static constexpr size_t kSlotP = (size_t)16 << (N + kCB);
  static constexpr size_t kSlot = kSlotP + (size_t)NR * 64 * 4;
  // ring depth: enough blocks in flight for the items the CTAs hold (152 x 3 buffers), within
  // about 48 MiB of L2
  static constexpr int NS = N <= 12 ? 6 : N == 13 ? 5 : 3;
  static_assert(NS <= kTiledSlots, "control block has room for the ring");
  // stage-2 items of block b follow stage-1 tiles of block b + LAG in the work order, so that
  // block b's tiles are finished by the time its stage-2 items are taken; a stage-1 tile of
  // block b reuses the slot of block b - NS, whose stage-2 items come LAG - NS + 1 <= -1 groups
  // earlier
  static constexpr int LAG = N <= 12 ? 3 : N == 13 ? 2 : 1;
  static_assert(NS >= LAG + 2, "slot reuse waits on items taken at least a group earlier");
  static constexpr size_t kWorkspace = kTiledCtrlBytes + NS * kSlot;
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
__device__ __forceinline__ void red_relaxed_add(int* p, int v) {
  asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
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
// 2D tensor tile (x = innermost coordinate, in the map's 8-byte elements; y = row)
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar), "l"(pol)
      : "memory");
}
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared state of one CTA.
struct Shared {
  uint64_t full[kBufs];   // buffer filled: producer arrival + copied bytes
  uint64_t empty[kBufs];  // buffer released: one arrival per consumer warp
  uint64_t done[kBufs];   // item's stores issued: one arrival per consumer warp (release warp waits)
  int item[kBufs];        // work item in the buffer, -1 = no more work
  int rel_slot[kBufs];    // per buffer use: slot to publish (stage 1), -1 (stage 2), -2 (end)
  int ok[2];              // per consumer group: its next buffer arrived (broadcast by its thread 0)
  int waited_use[kBufs];  // per buffer: the last use whose data a consumer group waited for
  int issued_use[kBufs];  // per buffer: the last use whose copies the producer issued
  int released;           // buffer uses the release warp has handled
  uint32_t smax[2][64];   // stage 1, per group: (use + 1) << 11 | largest exponent of each class
};

// Named barrier of one consumer group (ID 1 + group, THREADS threads).
template <int THREADS>
struct GroupBar {
  uint32_t id;
  __device__ __forceinline__ void sync() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(THREADS) : "memory");
  }
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

// Work item -> (stage, block, index within the block). Group g of the order holds the
// stage-1 tiles of block g, then the stage-2 items of block g - LAG; false for the padding
// items (stage 1 past the last block, stage 2 before the first).
template <int N>
struct Item {
  bool s1;
  int b, j;
  __device__ __forceinline__ bool decode(int item, int blocks) {
    constexpr int group = Geo<N>::n1 + Geo<N>::n2;
    const int g = item / group, r = item % group;
    s1 = r < Geo<N>::n1;
    b = s1 ? g : g - Geo<N>::LAG;
    j = s1 ? r : r - Geo<N>::n1;
    return s1 ? g < blocks : b >= 0;
  }
};

__device__ __forceinline__ char* slot_base(TiledCtrl* ws, size_t slot_bytes, int s) {
  return reinterpret_cast<char*>(ws) + kTiledCtrlBytes + (size_t)s * slot_bytes;
}

// ---------------------------------------------------------------------- producer --
template <int N, class AR, int GROUPS>
__device__ void producer(const CUtensorMap* map, int count, TiledCtrl* ws, Shared& sh, uint32_t buf0) {
  using GE = Geo<N>;
  constexpr uint32_t D = 1u << N;
  constexpr int nb = 1 << (N - kCB);
  constexpr uint32_t kTileBytes = 64u * 64u * sizeof(typename AR::Raw);
  constexpr int kX = (int)sizeof(typename AR::Raw) / 8;  // map elements per matrix element
  const int lane = threadIdx.x & 31;
  const int blocks = nb * count;
  const int n_items = (blocks + GE::LAG) * (GE::n1 + GE::n2);
  const uint64_t pol_first = policy_evict_first();
  if (lane != 0) return;  // one thread drives the ring
  asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
  int next = atomicAdd(&ws->counter, 1);
  for (int use = 0;;) {
    const int item = next;
    const bool done = item >= n_items;
    Item<N> it;
    if (!done) {
      next = atomicAdd(&ws->counter, 1);  // its latency overlaps the rest of this item
      if (!it.decode(item, blocks)) continue;
    }
    const int buf = use % kBufs;
    const uint32_t full = smem_addr(&sh.full[buf]);
    if (use >= kBufs && !wait_phase(smem_addr(&sh.empty[buf]), ((use / kBufs) - 1) & 1, &ws->status))
      break;  // the consumers never released the buffer: they give up on their own wait
    bool ok = true;
    if (use == 0 && ws->stall) {  // test hook: wait (briefly) for a count nothing raises
      int i = 0;
      for (; i < kStallPolls && ld_acquire(&ws->stall) != 0x7FFFFFFF; ++i) __nanosleep(128);
      atomicExch(&ws->status, kStatusTimeout);
      ok = false;
    }
    const int s = done ? 0 : it.b % GE::NS, gen = done ? 0 : it.b / GE::NS;
    if (!done && ok) {  // dependencies: the slot must be free (stage 1) or complete (stage 2)
      if (it.s1) {
        if (gen > 0) ok = wait_count(&ws->s2_done[s], GE::n2 * gen, &ws->status);
      } else {
        ok = wait_count(&ws->s1_done[s], GE::n1 * (gen + 1), &ws->status);
        // the chunk was written through the generic proxy; the copy reads it through the async one
        asm volatile("fence.proxy.async.global;" ::: "memory");
      }
    }
    if (done || !ok) {  // no more work (or a dependency never came): one end mark per group
      sh.item[buf] = -1;
      mbar_arrive(full);
      for (int g = 1; g < GROUPS; ++g) {
        const int u = use + g, b = u % kBufs;
        if (u >= kBufs && !wait_phase(smem_addr(&sh.empty[b]), ((u / kBufs) - 1) & 1, &ws->status)) break;
        sh.item[b] = -1;
        mbar_arrive(smem_addr(&sh.full[b]));
      }
      break;
    }
    const uint32_t dst = buf0 + (uint32_t)(buf * GE::kBuf);
    sh.item[buf] = item;
    if (it.s1) {
      mbar_arrive_tx(full, kTileBytes);
      const uint32_t k = (uint32_t)(it.b % nb), row0 = (uint32_t)it.j << kTB;
      const uint32_t colb = (row0 ^ (k << kCB)) & ~63u;
      tma_2d(dst, map, (int)colb * kX, (int)((uint32_t)(it.b / nb) * D + row0), full, pol_first);
    } else {
      mbar_arrive_tx(full, (uint32_t)(GE::kChunk + GE::kEOct + 32));
      const uint32_t o = (uint32_t)it.j & 7u, q = (uint32_t)it.j >> 3;
      char* sb = slot_base(ws, GE::kSlot, s);
      bulk_g2s(dst, sb + (size_t)(o * GE::NQ + q) * GE::kChunk, (uint32_t)GE::kChunk, full, pol_first);
      bulk_g2s(dst + (uint32_t)GE::kChunk, sb + GE::kSlotP + (size_t)o * GE::kEOct, (uint32_t)GE::kEOct, full,
               pol_first);
      bulk_g2s(dst + (uint32_t)(GE::kChunk + GE::kEOct), &ws->emax[s][o * 8], 32u, full, pol_first);
    }
    sh.issued_use[buf] = use;
    ++use;
  }
}

// ------------------------------------------------------------------- release warp --
// Publishes finished stage-1 tiles, in the consumers' order (one thread).
__device__ void releaser(TiledCtrl* ws, Shared& sh) {
  if ((threadIdx.x & 31) != 0) return;
  volatile int* released = &sh.released;
  for (int use = 0;; ++use) {
    const int buf = use % kBufs;
    if (!wait_phase(smem_addr(&sh.done[buf]), (use / kBufs) & 1, &ws->status)) break;
    const int r = sh.rel_slot[buf];
    if (r == -2) break;
    // every consumer warp's stores precede its arrival; the release makes them visible first
    if (r >= 0) red_release_add(&ws->s1_done[r], 1);
    __threadfence_block();  // the read of rel_slot[buf] completes before its slot may be rewritten
    *released = use + 1;
  }
}

// ---------------------------------------------------------------------- stage 1 --
// Per-thread constants of the stage-1 layout (computed once per thread).
template <int RB, int N>
struct S1Thread {
  using LY = Layout<kUB, kTB, RB>;
  uint32_t c;       // class within the block
  uint32_t ld;      // 16-byte slot of the thread's register-0 element in the tile: (i << 6) | (i ^ c)
  uint32_t xw, xr;  // swizzled exchange slots (write at phase 0, read at phase 1)
  uint32_t st;      // scratch entry of the thread's register-0 output, without the tile offset
  __device__ __forceinline__ void init(uint32_t t) {
    using GE = Geo<N>;
    constexpr int LAST = LY::NPH - 1;
    static_assert(LY::NPH == 2, "one exchange");
    c = t & 63u;
    const uint32_t it = LY::thread_u(0, t) >> kCB;
    ld = (it << 6) | (it ^ c);
    const uint32_t u0 = LY::thread_u(0, t), u1 = LY::thread_u(1, t);
    xw = u0 ^ swz_term(u0);
    xr = u1 ^ swz_term(u1);
    const uint32_t wt = LY::thread_u(LAST, t) >> kCB;
    st = (c >> 3) * GE::NQ * (uint32_t)(GE::kChunk / 16) + (c & 7u) + (wt >> GE::ZB) * (uint32_t)(GE::kChunk / 16) +
         ((wt & ((1u << GE::ZB) - 1u)) << 3);
  }
};

// Register j's offset from the thread's register-0 entry (compile-time).
template <class LY, int N>
__host__ __device__ constexpr uint32_t s1_store_off(int j) {
  using GE = Geo<N>;
  const uint32_t w = LY::reg_u(LY::NPH - 1, j) >> kCB;
  return (w >> GE::ZB) * (uint32_t)(GE::kChunk / 16) + ((w & ((1u << GE::ZB) - 1u)) << 3);
}
template <class LY>
__host__ __device__ constexpr uint32_t s1_load_off(int j) {
  const uint32_t i = LY::reg_u(0, j) >> kCB;
  return (i << 6) | i;  // XORed into the thread's slot (the bits are the thread's zero bits)
}

// Tile R of block k in the buffer: element (i, c) at slot (i << 6) | (i ^ c).
template <int N, int RB, class AR, int CT>
__device__ __forceinline__ void stage1(uint32_t tile, const S1Thread<RB, N>& th, uint32_t tg, const GroupBar<CT>& bar,
                                       char* slot, TiledCtrl* ws, int s, int gen, uint32_t R, uint32_t* smax,
                                       uint32_t tag, uint64_t pol_keep) {
  using GE = Geo<N>;
  using LY = Layout<kUB, kTB, RB>;
  static_assert(LY::K == kCB, "tile = 64 classes x 64 rows");
  constexpr int E = LY::E;
  constexpr uint32_t kEs = sizeof(typename AR::Raw);
  typename AR::Raw raw[E];
  uint32_t emax = 0;
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const uint32_t a = tile + (th.ld ^ s1_load_off<LY>(j)) * kEs;
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
    atomicMax(&smax[th.c], (tag << 11) | (emax >> 20));  // older tags are smaller: no reset needed
  }
  bar.sync();  // exponents complete, and every tile read is done: the buffer serves the exchange
  if constexpr (AR::kScaled) Ekey = (smax[th.c] & 0x7FFu) << 20;
  const typename AR::Conv cv = AR::make_conv(N, Ekey, 0);
  typename AR::Elem v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = AR::template convert<0>(raw[j], cv, 0u);
  wht_regs<AR, LY::gcount(0), E>(v);
  // exchange phase 0 -> 1 (the barrier above already ended the reads of the tile)
#pragma unroll
  for (int j = 0; j < E; ++j)
    sts128(tile + 16u * (th.xw ^ (LY::reg_u(0, j) ^ swz_term(LY::reg_u(0, j)))), AR::pack(v[j]));
  bar.sync();
#pragma unroll
  for (int j = 0; j < E; ++j)
    v[j] = AR::unpack(lds128(tile + 16u * (th.xr ^ (LY::reg_u(1, j) ^ swz_term(LY::reg_u(1, j))))));
  wht_regs<AR, LY::gcount(1), E>(v);
  // P[o][q][R][wl][c8]
  uint4* P = reinterpret_cast<uint4*>(slot) + th.st + (R << (GE::ZB + 3));
#pragma unroll
  for (int j = 0; j < E; ++j) st_hint(P + s1_store_off<LY, N>(j), AR::pack(v[j]), pol_keep);
  if (tg < 64) {
    uint32_t* Ep = reinterpret_cast<uint32_t*>(slot + GE::kSlotP);
    Ep[((tg >> 3) * GE::NR + R) * 8 + (tg & 7u)] = Ekey;
    if constexpr (AR::kScaled) red_max(&ws->emax[s][tg], ((uint32_t)(gen + 1) << 11) | (Ekey >> 20));
  }
}

// ---------------------------------------------------------------------- stage 2 --
template <int RB, int N>
struct S2Thread {
  using LY = Layout<kUB, Geo<N>::L, RB>;
  static constexpr int NPH = LY::NPH;
  uint32_t c8, wt;     // class within the octet, thread part of w (without the item's group)
  uint32_t u0;         // thread part of the element index at phase 0
  uint32_t ex[2 * (NPH - 1)];  // swizzled exchange slots: write/read per exchange
  uint32_t ht;         // thread part of h at the last phase
  __device__ __forceinline__ void init(uint32_t t) {
    constexpr int ZB = Geo<N>::ZB;
    c8 = t & 7u;
    wt = (t >> 3) & ((1u << ZB) - 1u);
    u0 = LY::thread_u(0, t);
#pragma unroll
    for (int p = 0; p + 1 < NPH; ++p) {
      const uint32_t a = LY::thread_u(p, t), b = LY::thread_u(p + 1, t);
      ex[2 * p] = a ^ swz_term(a);
      ex[2 * p + 1] = b ^ swz_term(b);
    }
    ht = LY::thread_u(NPH - 1, t) >> LY::K;
  }
};

template <class LY, class AR, class BAR, int P>
__device__ __forceinline__ void s2_phases(typename AR::Elem (&v)[LY::E], uint32_t xaddr, const uint32_t* ex,
                                          const BAR& bar) {
  wht_regs<AR, LY::gcount(P), LY::E>(v);
  if constexpr (P + 1 < LY::NPH) {
    bar.sync();  // previous reads of the buffer are done
#pragma unroll
    for (int j = 0; j < LY::E; ++j)
      sts128(xaddr + 16u * (ex[2 * P] ^ (LY::reg_u(P, j) ^ swz_term(LY::reg_u(P, j)))), AR::pack(v[j]));
    bar.sync();
#pragma unroll
    for (int j = 0; j < LY::E; ++j)
      v[j] = AR::unpack(lds128(xaddr + 16u * (ex[2 * P + 1] ^ (LY::reg_u(P + 1, j) ^ swz_term(LY::reg_u(P + 1, j))))));
    s2_phases<LY, AR, BAR, P + 1>(v, xaddr, ex, bar);
  }
}

// Item j = (o, q) of block k: the chunk holds entry (R, wl, c8) at 16-byte slot
// (R << K2) | (wl << 3) | c8 -- the unit's own element order -- then E[R][c8], then the
// eight tagged class maxima.
template <int N, int RB, class AR, int CT>
__device__ __forceinline__ void stage2(uint32_t chunk, const char* chunk_gen, const S2Thread<RB, N>& th,
                                       const GroupBar<CT>& bar, void* __restrict__ out, unsigned long long obase,
                                       uint32_t k, uint32_t item, uint64_t pol_out) {
  using GE = Geo<N>;
  using LY = Layout<kUB, GE::L, RB>;
  constexpr int K = LY::K, E = LY::E, LAST = LY::NPH - 1, ZB = GE::ZB;
  static_assert(K == GE::K2, "stage-2 unit = 8 classes x 2^ZB w x 2^L row blocks");
  const uint32_t o = item & 7u, q = item >> 3;
  const uint32_t w = (q << ZB) | th.wt;
  const uint32_t x = (k << kCB) | (o << 3) | th.c8;
  typename AR::Elem v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = AR::unpack(lds128(chunk + 16u * (th.u0 + LY::reg_u(0, j))));
  typename AR::Conv cv;
  if constexpr (AR::kScaled) {
    const uint32_t* Es = reinterpret_cast<const uint32_t*>(chunk_gen + GE::kChunk);
    const int em = (int)(Es[GE::NR * 8 + th.c8] & 0x7FFu);
    cv = AR::make_conv(N, (uint32_t)em << 20, -N);
    if (!cv.nan) {
      const uint32_t* Et = Es + (((th.u0 >> K) << 3) | th.c8);
#pragma unroll
      for (int j = 0; j < E; ++j) {
        // tile at exponent et was converted at scale 2^(s + em - et): shift right by em - et
        // (all-zero tiles have et = 0 and hold zeros)
        AR::align(v[j], min(em - (int)(Et[(LY::reg_u(0, j) >> K) << 3] >> 20), 63));
      }
    }
  } else {
    cv = AR::make_conv(N, 0u, -N);
  }
  s2_phases<LY, AR, GroupBar<CT>, 0>(v, chunk, th.ex, bar);  // the first barrier also ends the chunk reads
  // c(x, z), z = (h << 6) | w, h = ht | (register part)
  Addr<N, false> ao;
  ao.init(obase, x, (th.ht << kTB) | w);
  constexpr int p0 = LY::regrow(LAST, 0) < 0 ? -1 : LY::regrow(LAST, 0) + kTB;
  constexpr int p1 = LY::regrow(LAST, 1) < 0 ? -1 : LY::regrow(LAST, 1) + kTB;
  constexpr int p2 = LY::regrow(LAST, 2) < 0 ? -1 : LY::regrow(LAST, 2) + kTB;
  constexpr int p3 = LY::regrow(LAST, 3) < 0 ? -1 : LY::regrow(LAST, 3) + kTB;
  BitSum<p0, p1, p2, p3> xo;
  xo.init(x);
  const uint32_t ko = (uint32_t)__popc(x & ((th.ht << kTB) | w));
#pragma unroll
  for (int j = 0; j < E; ++j)
    AR::store_hint(out, ao.at((LY::reg_u(LAST, j) >> K) << kTB), v[j], cv, ko + xo.at(j), pol_out);
}

// ---------------------------------------------------------------------- consumers --
// Consumer group `g` (CT threads) takes the buffer uses g, g + GROUPS, g + 2 GROUPS, ...
template <int N, int RB, class AR, int CT, int GROUPS>
__device__ void consumer(void* __restrict__ out, int count, TiledCtrl* ws, Shared& sh, char* bufs, uint32_t buf0) {
  using GE = Geo<N>;
  constexpr uint32_t D = 1u << N;
  constexpr int nb = 1 << (N - kCB);
  const uint32_t g = threadIdx.x / CT, tg = threadIdx.x % CT, lane = threadIdx.x & 31u;
  const GroupBar<CT> bar{1u + g};
  const int blocks = nb * count;
  const uint64_t pol_keep = policy_evict_last(), pol_first = policy_evict_first();
  S1Thread<RB, N> t1;
  S2Thread<RB, N> t2;
  t1.init(tg);
  t2.init(tg);
  volatile int* released = &sh.released;
  int use = (int)g;
  for (;; use += GROUPS) {
    const int buf = use % kBufs;
    const uint32_t full = smem_addr(&sh.full[buf]);
    const uint32_t parity = (use / kBufs) & 1;
    // the group's thread 0 waits (bounded) and broadcasts, so that the group leaves together;
    // it also keeps the release warp less than a ring behind (its barrier phases must not be
    // lapped, and it reads rel_slot[] of the use a ring earlier)
    if (tg == 0) {
      bool ok = true;
      for (int i = 0; *released < use - kBufs + 1; ++i) {
        if (i == kPolls) {
          atomicExch(&ws->status, kStatusTimeout);
          ok = false;
          break;
        }
        __nanosleep(64);
      }
      __threadfence_block();  // the release warp's read of rel_slot[] precedes this group's write of it
      ok = ok && wait_phase(full, parity, &ws->status);
      if (ok) sh.waited_use[buf] = use;
      sh.ok[g] = ok;
    }
    bar.sync();
    if (!sh.ok[g]) break;
    for (int i = 0; i < kPolls && !mbar_try_wait(full, parity); ++i) {  // completes at once: acquires the data
    }
    const int item = sh.item[buf];
    if (item < 0) break;
    Item<N> it;
    it.decode(item, blocks);
    const int s = it.b % GE::NS, gen = it.b / GE::NS;
    const uint32_t addr = buf0 + (uint32_t)(buf * GE::kBuf);
    if (tg == 0) sh.rel_slot[buf] = it.s1 ? s : -1;
    if (it.s1) {
      stage1<N, RB, AR, CT>(addr, t1, tg, bar, slot_base(ws, GE::kSlot, s), ws, s, gen, (uint32_t)it.j, sh.smax[g],
                            (uint32_t)use + 1u, pol_keep);
    } else {
      // the slot's data is in shared memory: a relaxed count suffices (the copy has completed)
      if (tg == 0) red_relaxed_add(&ws->s2_done[s], 1);
      stage2<N, RB, AR, CT>(addr, bufs + (size_t)buf * GE::kBuf, t2, bar, out,
                            (unsigned long long)(it.b / nb) * D * D, (uint32_t)(it.b % nb), (uint32_t)it.j, pol_first);
    }
    // this warp is done with the buffer and has issued its stores
    __syncwarp();
    if (lane == 0) {
      // the buffer was accessed through the generic proxy; the next copy writes it through the async one
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_addr(&sh.empty[buf]));
      mbar_arrive(smem_addr(&sh.done[buf]));
    }
  }
  // tell the release warp to stop: a done phase marked -2 (after the previous uses' phases,
  // which every warp of their groups has arrived on)
  const int buf = use % kBufs;
  if (tg == 0) sh.rel_slot[buf] = -2;
  bar.sync();
  if (lane == 0) mbar_arrive(smem_addr(&sh.done[buf]));
}

// 8 elements per thread: one group of 512 consumer threads; 16 per thread: two groups of
// 256, each on its own work item.
template <int RB>
struct TiledShape {
  static constexpr int kGroups = RB == 4 ? 2 : 1;
  static constexpr int kGroupThreads = 1 << (kUB - RB);
  static constexpr int kConsumers = kGroups * kGroupThreads;
  static constexpr int kGroupWarps = kGroupThreads / 32;
  static constexpr int kThreads = kConsumers + 64;  // + producer warp + release warp
};

template <int N, int RB, class AR>
__global__ void __launch_bounds__(TiledShape<RB>::kThreads, 1)
    tiled_kernel(const __grid_constant__ CUtensorMap map, void* __restrict__ out, int count, TiledCtrl* ws) {
  constexpr int CT = TiledShape<RB>::kGroupThreads;
  constexpr int GROUPS = TiledShape<RB>::kGroups;
  constexpr int CONSUMERS = TiledShape<RB>::kConsumers;
  extern __shared__ __align__(1024) char bufs[];
  __shared__ Shared sh;
  const uint32_t t = threadIdx.x;
  const uint32_t buf0 = smem_addr(bufs);
  if (t == 0) {
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(smem_addr(&sh.full[b]), 1);
      mbar_init(smem_addr(&sh.empty[b]), TiledShape<RB>::kGroupWarps);  // one use = one group
      mbar_init(smem_addr(&sh.done[b]), TiledShape<RB>::kGroupWarps);
      sh.waited_use[b] = -1;
      sh.issued_use[b] = -1;
    }
    sh.released = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (t < 128) sh.smax[t >> 6][t & 63] = 0;
  __syncthreads();
  if (t < (uint32_t)CONSUMERS) {
    consumer<N, RB, AR, CT, GROUPS>(out, count, ws, sh, bufs, buf0);
  } else if (t < (uint32_t)CONSUMERS + 32) {
    producer<N, AR, GROUPS>(&map, count, ws, sh, buf0);
    __syncwarp();  // lane 0 drove the ring alone; the barrier below wants whole warps
  } else {
    releaser(ws, sh);
    __syncwarp();
  }
  __syncthreads();
  // after a wait gave up: wait (bounded) for copies still landing in buffers nobody waited for
  if (t == (uint32_t)CONSUMERS) {
    for (int b = 0; b < kBufs; ++b) {
      const int u = sh.issued_use[b];
      if (u <= sh.waited_use[b]) continue;
      const uint32_t full = smem_addr(&sh.full[b]);
      for (int i = 0; i < kPolls && !mbar_try_wait(full, (u / kBufs) & 1); ++i) {
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
  CUtensorMap map;
  e = tiled_tensor_map(&map, G, N, count, (int)sizeof(typename AR::Raw));
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
  if (tiled_take_stall()) {
    e = cudaMemsetAsync(reinterpret_cast<char*>(ws) + offsetof(TiledCtrl, stall), 1, 1, st);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, TiledShape<RB>::kThreads, smem, st>>>(map, out, count, reinterpret_cast<TiledCtrl*>(ws));
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

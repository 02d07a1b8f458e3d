// twostage_impl.cuh -- the two-stage XOR-diagonal decomposition for 12 <= N <= 14 with
// warp-independent consumers (kernel and launcher templates; host side in tiled.cu,
// instantiations in twostage_*.cu).
//
// The transform of Eq. (13) for XY-mask x is split over the row index r = (R, i), R = r >> 6,
// i = r & 63, as in the block-tiled kernel: stage 1 transforms the 6 bits of i of a tile of
// 64 masks x 64 rows (the 64 x 64 submatrix of G at rows 64R.., columns (64R ^ 64k).., one 2D
// TMA load) and writes the partial sums to an L2-resident scratch ring; stage 2 transforms the
// L = N - 6 bits of R for every (mask, partial index w) and stores the coefficients.
//
// What differs: every consumer warp owns 512 elements of a work item and runs its whole part
// of the item alone -- loads, conversion, butterflies, one exchange through shared memory, and
// stores -- with __syncwarp as its only synchronisation; no named barrier ties the warps of an
// item together, so warps overlap each other's memory, shared-memory and integer phases.
//  - stage 1: warp o of the item takes the masks 8o..8o+7 (an octet) of the tile. Each lane
//    holds one mask and 16 rows (four row bits in registers, two in the lane); the exponent
//    maximum of a mask over the tile is a two-step shuffle; four butterfly stages run in
//    registers, the exchange writes the values back into the slots the warp read (the warp's
//    own part of the tile) and reads them in the second layout, and two more stages finish the
//    six. Complex64 tiles hold 8-byte elements: the 16-byte values cross in two rounds.
//  - stage 2: a work item is one 64 KiB chunk of the scratch -- all 2^L tiles of 2^(12-L)
//    transforms -- and warp p reads its 2^(9-L) transforms x 2^L tiles with its own 2D TMA box
//    into its own 8 KiB of the buffer; four stages in registers, an in-place exchange with an
//    XOR swizzle that keeps both access patterns free of bank conflicts, the remaining L - 4
//    stages, the phase, the scale and the stores of c(x, z).
// Scratch layout of a slot (one block of 64 masks): P[chunk jj][R][t] (chunk jj = o (2^(L-3)) +
// (w >> (9-L)), transform t = ((w mod 2^(9-L)) << 3) | c8 for mask 8o + c8 and stage-1 output
// index w), then, after every slot's P, E[slot][o][R][c8] (the exponent key of each mask in each
// tile). Entries are 16 bytes for complex128 (the int64 pair; stage-1 stores are 128- or 256-byte
// runs of one (chunk, R)) and 8 bytes for complex64 (each part's compensated pair rounded once
// to a float: half the ring's bytes and L2 traffic; both stages still sum with compensation).
//
// Schedule, dependencies and bounded waits are those of the block-tiled kernel: one persistent
// CTA per SM; a copy warp takes work items from a global counter in the order S1(block 0) ..
// S1(LAG), S2(0), S1(LAG + 1), S2(1), ..., waits (bounded, acquire loads) for each item's
// dependencies and fills a 3-deep ring of shared-memory buffers; two teams of 8 consumer warps
// take alternate buffers; a release warp publishes each finished stage-1 tile with a release
// reduction. Every item waited on was taken from the counter earlier, and an item whose copies
// were issued is finished by its consumers without waiting on any other item, so every wait
// ends; each wait is bounded nevertheless and records PAULI_ERR_TIMEOUT when it gives up.
// Registers: the consumer warpgroups raise their budget to 112 per thread (setmaxnreg) with the
// registers the copy/release warpgroup gives up.
#pragma once
#include <cuda.h>

#include <cstddef>

#include <type_traits>

#include "c64x.cuh"
#include "kernels.h"
#include "ptx.cuh"
#include "tiled.h"
#include "xordiag_impl.cuh"

namespace pauli {

cudaError_t tiled_workspace(cudaStream_t st, size_t bytes, void** out);
cudaError_t tiled_tensor_map(CUtensorMap* map, const void* G, int N, int count, int elem);
// `rows` rows of 2^wlog elements (a shard's block-XOR layout), 64 x 64 boxes (tiled.cu).
cudaError_t tiled_tensor_map_rows(CUtensorMap* map, const void* G, int wlog, long long rows, int elem);
// 4D map of the scratch ring's stage-2 chunks (tiled.cu).
cudaError_t scratch_tensor_map4(CUtensorMap* map, void* base, int chunks, int nr, int slice_words);
bool tiled_take_stall();

namespace ts {
namespace {
using namespace xd;
using namespace ptx;

constexpr int kCB = 6;  // masks per block: 2^6
constexpr int kTB = 6;  // rows per stage-1 tile: 2^6
constexpr int kBufs = 3;
constexpr int kRel = 6;  // ring of the release warp's records: uses in flight between the teams' stores and its publishing
constexpr int kTeams = 2, kTeamWarps = 8, kConsumerWarps = kTeams * kTeamWarps;
constexpr int kThreads = (kConsumerWarps + 4) * 32;  // + a warpgroup of copy, release and 2 idle warps
constexpr int kConsumerRegs = 112, kHelperRegs = 32;
static_assert(kConsumerWarps * 32 * kConsumerRegs + 128 * kHelperRegs <= kThreads * 96,
              "the register split fits the launch's 96 registers per thread");
constexpr int kStatusTimeout = 8;     // PAULI_ERR_TIMEOUT
constexpr int kStallPolls = 1 << 15;  // the test hook's wait: well under a second

// Bytes of one scratch entry: complex128 stage-1 values are int64 pairs (16 bytes); complex64
// values are stored as one float per part, the compensated pair (hi, lo) rounded once (8 bytes).
template <class AR>
constexpr int kScratchEntry = std::is_base_of<ArC64X, AR>::value ? 8 : 16;

template <int N, int SE = 16>
struct Geo {
  static constexpr int L = N - kTB;      // stage-2 bits
  static constexpr int NR = 1 << L;      // tiles per block = stage-2 items per block
  static constexpr int TPI = 4096 >> L;  // transforms per stage-2 item
  static constexpr int TPW = TPI / 8;    // transforms per warp = w values per chunk and mask
  static constexpr int LTPW = 9 - L;     // log2 TPW
  static constexpr int RLB = L - 4;      // tile bits in the lanes at stage 2's first phase
  static constexpr int NCH = NR / 8;     // chunks per octet
  static_assert(SE == 8 || SE == 16, "scratch entries of 8 or 16 bytes");
  static constexpr size_t kChunk = 4096 * SE;  // bytes of one chunk in the scratch and of its copy
  static constexpr uint32_t kSlice = 512 * SE;  // one consumer warp's part of a chunk copy
  // a buffer's chunk area: 4096 16-byte entries (the stage-2 exchange runs on 16-byte entries;
  // with 8-byte scratch entries warp p's exchange uses its own copied slice and the slice's
  // twin in the area's upper half)
  static constexpr size_t kChunkArea = 65536;
  static constexpr size_t kSlotP = (size_t)NR * kChunk;
  static constexpr size_t kSlotE = (size_t)NR * 64 * 4;
  static constexpr size_t kEOct = (size_t)NR * 8 * 4;
  static constexpr size_t kBuf = kChunkArea + kEOct + 128;
  // ring depth and lag, measured: 13 x 4 MiB with a lag of 6 blocks at N = 12 (0.163 ms against
  // 0.180 ms with 6 slots and a lag of 3), 6 x 8 MiB / 3 at N = 13, 4 x 16 MiB / 2 at N = 14 (deeper
  // rings spill from L2 there and are slower)
  static constexpr int NS = N <= 12 ? 13 : N == 13 ? 6 : 4;
  // stage-2 items of block b follow stage-1 tiles of block b + LAG in the work order
  static constexpr int LAG = N <= 12 ? 6 : N == 13 ? 3 : 2;
  static_assert(NS <= kTiledSlots, "control block has room for the ring");
  static_assert(NS >= LAG + 2, "slot reuse waits on items taken at least a group earlier");
  static constexpr size_t kPBase = kTiledCtrlBytes;
  static constexpr size_t kEBase = kTiledCtrlBytes + NS * kSlotP;
  static constexpr size_t kWorkspace = kEBase + NS * kSlotE;
  static constexpr int n1 = NR, n2 = NR;
  static_assert(L >= 6 && L <= 8, "12 <= N <= 14");
};

// Stage-1 bit assignment of a warp's 512 elements (mask c8 in lane bits 0..2, row / output bits
// u0..u5): in phase A lane bits 3, 4 hold row bits A0, A1 and register bit k holds row bit ra(k);
// in phase B lane bits 3, 4 hold output bits B0 = 0, B1 = 1 and register bit k holds bit rb(k)
// (bits 0, 1 of the register index: the two row bits left to transform). The tile holds element
// (u, c) at slot 64 u + (u ^ c); the exchange puts element u at the slot of row xrow(u).
//  16-byte elements (one 128-byte wavefront per 8-lane quarter): A = (4, 5); the bank group of a
//    slot is (u ^ c) & 7, which the quarter's 8 masks make distinct in every phase.
//  8-byte elements (one wavefront per 16-lane half): A = (3, 4) so that the half's lanes cover
//    bit 3 of the row as well, and xrow(u) = u ^ (u0 << 3) makes bit 3 of the exchange row vary
//    with the lane bit B0 in phase B.
template <int ES>
struct S1Bits;
template <>
struct S1Bits<16> {
  static constexpr int A0 = 4, A1 = 5, B0 = 0, B1 = 1;
  __host__ __device__ static constexpr int ra(int k) { return k; }                  // 0, 1, 2, 3
  __host__ __device__ static constexpr int rb(int k) { return k < 2 ? 4 + k : k; }  // 4, 5, 2, 3
  __host__ __device__ static constexpr uint32_t xrow(uint32_t u) { return u; }
};
template <>
struct S1Bits<8> {
  static constexpr int A0 = 3, A1 = 4, B0 = 0, B1 = 1;
  __host__ __device__ static constexpr int ra(int k) { return k < 3 ? k : 5; }      // 0, 1, 2, 5
  __host__ __device__ static constexpr int rb(int k) { return k < 2 ? 3 + k : k == 2 ? 2 : 5; }  // 3, 4, 2, 5
  __host__ __device__ static constexpr uint32_t xrow(uint32_t u) { return u ^ ((u & 1u) << 3); }
};
template <class SB>
__host__ __device__ constexpr uint32_t reg_a(int j) {
  uint32_t u = 0;
  for (int k = 0; k < 4; ++k)
    if ((j >> k) & 1) u |= 1u << SB::ra(k);
  return u;
}
template <class SB>
__host__ __device__ constexpr uint32_t reg_b(int j) {
  uint32_t u = 0;
  for (int k = 0; k < 4; ++k)
    if ((j >> k) & 1) u |= 1u << SB::rb(k);
  return u;
}
// Slot of row v's element of mask c: 64 v + (v ^ c). Linear over GF(2) in v for fixed c once
// the mask's part is factored out: slot(v_lane ^ v_reg) = slot(v_lane) ^ sreg(v_reg).
__host__ __device__ constexpr uint32_t sreg(uint32_t v) { return (v << 6) | v; }

// Scratch entry offset (16-byte units, within the slot's P) of output index w for the given
// mask c8 = 0 and tile R = 0: linear in the bits of w (chunk part and transform part).
template <int N>
__host__ __device__ constexpr uint32_t s1_w_off(uint32_t w) {
  using GE = Geo<N>;
  return (w >> GE::LTPW) * (uint32_t)(GE::NR * GE::TPI) + ((w & (GE::TPW - 1u)) << 3);
}

// The complex64 policy re-splits stage-1 values on each mask's grid in stage 2 (c64x.cuh) instead
// of shifting fixed-point tiles; its exponent keys are float exponent fields.
template <class AR>
constexpr bool kRegrid = std::is_base_of<ArC64X, AR>::value;
template <class AR>
__device__ __forceinline__ uint32_t key_exp(uint32_t key) {
  if constexpr (kRegrid<AR>) return key >> 23;
  return key >> 20;
}
template <class AR>
__device__ __forceinline__ uint32_t exp_to_key(uint32_t e) {
  if constexpr (kRegrid<AR>) return e << 23;
  return e << 20;
}

// Work item -> (stage, block, index within the block).
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

struct Shared {
  uint64_t full[kBufs];   // producer arrival + copied bytes
  uint64_t empty[kBufs];  // one arrival per consumer warp of the team
  uint64_t done[kRel];    // use u % kRel: one arrival per warp of the team once its stores are issued
  int item[kBufs];        // work item in the buffer, -1 = no more work
  int use_of[kBufs];      // the buffer use whose copies `full` tracks (written before the arrival)
  int rel_slot[kRel];     // use u % kRel -- stage 1: slot to publish; -1 stage 2; -2 end of work
  int waited_use[kBufs];  // last use whose copies a consumer waited for
  int issued_use[kBufs];  // last use whose copies the producer issued
  int released;           // buffer uses the release warp has handled
};

// Every wait gives up after kWaitNs of wall time (the global timer), records PAULI_ERR_TIMEOUT
// and returns false; a launch takes milliseconds, so a wait that long means the results are lost.
constexpr unsigned long long kWaitNs = 1000000000ull;
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity, int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = now_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (now_ns() - t0 > kWaitNs) break;
  }
  atomicExch(status, kStatusTimeout);
  return false;
}
// Wait for the phase of buffer use `use`: parity complete and the buffer's use tag equal to it.
__device__ __forceinline__ bool wait_use(uint32_t bar, uint32_t parity, const int* tag, int use, int* status) {
  const volatile int* t = tag;
  if (mbar_try_wait(bar, parity) && *t == use) return true;
  const unsigned long long t0 = now_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity) && *t == use) return true;
    if (now_ns() - t0 > kWaitNs) break;
  }
  atomicExch(status, kStatusTimeout);
  return false;
}
__device__ __forceinline__ bool wait_count(const int* counter, int target, int* status) {
  if (ld_acquire(counter) >= target) return true;
  const unsigned long long t0 = now_ns();
  while (now_ns() - t0 <= kWaitNs) {
    if (ld_acquire(counter) >= target) return true;
    __nanosleep(128);
  }
  atomicExch(status, kStatusTimeout);
  return false;
}
// The copy warp's wait for the release warp: it then overwrites rel_slot[] of the released use, so
// the observation is ordered before those writes.
__device__ __forceinline__ bool wait_released(const volatile int* released, int target, int* status) {
  if (*released >= target) {
    __threadfence_block();
    return true;
  }
  const unsigned long long t0 = now_ns();
  while (now_ns() - t0 <= kWaitNs) {
    if (*released >= target) {
      __threadfence_block();
      return true;
    }
    __nanosleep(64);
  }
  atomicExch(status, kStatusTimeout);
  return false;
}

// The matrix, or one x-class shard of it (pauli_decompose_xhi): the 2^k stacked blocks of the
// block-XOR layout (2^N rows of 2^m elements, m = N - k) in, the coefficients of the classes
// x = xhi | x_lo out, compacted to (z_hi << 2m) | n_lo. The whole matrix is m = N, xhi = 0.
struct ShardArgs {
  int m;
  uint32_t xhi;
};
// Kernel modes: the whole matrix, one x-class shard, a Hermitian matrix read from its upper
// triangle (a tile below the diagonal is loaded from its mirror above and read transposed and
// conjugated; the diagonal tiles mirror their own lower halves; diagonal entries count with
// their real parts only).
constexpr int kWhole = 0, kShard = 1, kUpper = 2;

// ---------------------------------------------------------------------- copy warp --
template <int N, class AR, int MODE>
__device__ void producer(const CUtensorMap* gmap, const CUtensorMap* smap, int count, TiledCtrl* ws, Shared& sh,
                         uint32_t buf0, ShardArgs sa) {
  using GE = Geo<N, kScratchEntry<AR>>;
  constexpr uint32_t D = 1u << N;
  const int nbl = (MODE == kShard) ? sa.m - kCB : N - kCB, nb = 1 << nbl;  // mask blocks of 64 classes per matrix (or shard)
  const uint32_t wmask = (MODE == kShard) ? (1u << sa.m) - 1u : ~0u;
  constexpr uint32_t kTileBytes = 64u * 64u * sizeof(typename AR::Raw);
  constexpr int kX = (int)sizeof(typename AR::Raw) / 8;  // map words per matrix element
  const int blocks = nb * count;
  const int n_items = (blocks + GE::LAG) * (GE::n1 + GE::n2);
  const uint64_t pol_first = policy_evict_first();
  const volatile int* released = &sh.released;
  char* const E0 = reinterpret_cast<char*>(ws) + GE::kEBase;
  prefetch_tensormap(gmap);
  prefetch_tensormap(smap);
  // the last dependency this thread saw satisfied, per kind: (block + 1), 0 = none. Items come
  // in runs of one block; once an acquire load has seen a block's count, this thread's later
  // accesses are ordered after it, so the rest of the run needs no load.
  int seen1 = 0, seen2 = 0;
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
    // the team's warps have left the buffer, and the release warp has handled use - kRel
    if (use >= kBufs && !wait_phase(smem_addr(&sh.empty[buf]), ((use / kBufs) - 1) & 1, &ws->status)) break;
    if (use >= kRel && !wait_released(released, use - kRel + 1, &ws->status)) break;
    bool ok = true;
    if (use == 0 && ws->stall) {  // test hook: wait (briefly) for a count nothing raises
      for (int i = 0; i < kStallPolls && ld_acquire(&ws->stall) != 0x7FFFFFFF; ++i) __nanosleep(128);
      atomicExch(&ws->status, kStatusTimeout);
      ok = false;
    }
    const int s = done ? 0 : it.b % GE::NS, gen = done ? 0 : it.b / GE::NS;
    if (!done && ok) {  // the slot must be free (stage 1) or complete (stage 2)
      if (it.s1) {
        if (gen > 0 && seen1 != it.b + 1) {
          ok = wait_count(&ws->s2_done[s], GE::n2 * gen, &ws->status);
          seen1 = it.b + 1;
        }
      } else {
        if (seen2 != it.b + 1) {
          ok = wait_count(&ws->s1_done[s], GE::n1 * (gen + 1), &ws->status);
          seen2 = it.b + 1;
          fence_proxy_async_global();  // written through the generic proxy, read through the async one
        }
      }
    }
    if (done || !ok) {  // one end mark per team
      for (int g = 0; g < kTeams; ++g) {
        const int u = use + g, b = u % kBufs;
        if (g > 0) {
          if (u >= kBufs && !wait_phase(smem_addr(&sh.empty[b]), ((u / kBufs) - 1) & 1, &ws->status)) break;
          if (u >= kRel && !wait_released(released, u - kRel + 1, &ws->status)) break;
        }
        sh.item[b] = -1;
        sh.rel_slot[u % kRel] = -2;
        sh.use_of[b] = u;
        mbar_arrive(smem_addr(&sh.full[b]));
      }
      break;
    }
    const uint32_t full = smem_addr(&sh.full[buf]);
    const uint32_t dst = buf0 + (uint32_t)(buf * GE::kBuf);
    sh.item[buf] = item;
    sh.rel_slot[use % kRel] = it.s1 ? s : -1;
    sh.use_of[buf] = use;
    if (it.s1) {
      mbar_arrive_tx(full, kTileBytes);
      const uint32_t k = (uint32_t)(it.b & (nb - 1)), row0 = (uint32_t)it.j << kTB;
      const uint32_t colb = (row0 ^ (k << kCB)) & wmask & ~63u;  // column of the row's block (shard: in it)
      const uint32_t mrow = (uint32_t)(it.b >> nbl) * D;
      if (MODE == kUpper && colb < row0)  // below the diagonal: the mirror tile, read transposed
        tma_2d(dst, gmap, (int)row0 * kX, (int)(mrow + colb), full, pol_first);
      else
        tma_2d(dst, gmap, (int)colb * kX, (int)(mrow + row0), full, pol_first);
    } else {
      mbar_arrive_tx(full, (uint32_t)(GE::kChunk + GE::kEOct + 32));
      // one 4D box: the 8 warps' transform groups x all tiles of chunk j, warp slices contiguous
      tma_4d(dst, smap, 0, 0, 0, s * GE::NR + it.j, full, pol_first);
      const int o = it.j / GE::NCH;
      bulk_g2s(dst + (uint32_t)GE::kChunkArea, E0 + (size_t)s * GE::kSlotE + (size_t)o * GE::kEOct,
               (uint32_t)GE::kEOct, full, pol_first);
      bulk_g2s(dst + (uint32_t)(GE::kChunkArea + GE::kEOct), &ws->emax[s][o * 8], 32u, full, pol_first);
    }
    sh.issued_use[buf] = use;
    ++use;
  }
}

// ------------------------------------------------------------------- release warp --
__device__ void releaser(TiledCtrl* ws, Shared& sh) {
  volatile int* released = &sh.released;
  volatile int* rel = sh.rel_slot;
  for (int use = 0;; ++use) {
    const int q = use % kRel;
    if (!wait_phase(smem_addr(&sh.done[q]), (use / kRel) & 1, &ws->status)) break;
    const int r = rel[q];
    // every warp's stores precede its arrival; the release makes them visible first
    if (r >= 0) red_release_add(&ws->s1_done[r], 1);
    // the read of rel_slot[buf] is complete before the copy warp may learn that it can overwrite it
    __threadfence_block();
    *released = use + 1;
    if (r == -2) break;
  }
}

// ---------------------------------------------------------------------- stage 1 --
// e -> -e where the lane mask m is all ones, e unchanged where it is zero (exact: fixed-point
// values stay below 2^62 in magnitude, and a float changes only its sign bit).
__device__ __forceinline__ void negate_where(ArC128::Elem& e, uint32_t m) {
  const long long mm = (long long)(int)m;
  e.re = (e.re ^ mm) - mm;
  e.im = (e.im ^ mm) - mm;
}
__device__ __forceinline__ void negate_where(ArC64::Elem& e, uint32_t m) {
  const uint32_t sb = m & 0x80000000u;
  e.rh = __uint_as_float(__float_as_uint(e.rh) ^ sb);
  e.rl = __uint_as_float(__float_as_uint(e.rl) ^ sb);
  e.ih = __uint_as_float(__float_as_uint(e.ih) ^ sb);
  e.il = __uint_as_float(__float_as_uint(e.il) ^ sb);
}

// Warp o of a stage-1 item: masks 8o..8o+7 of the tile at `tile` (element (i, col) at slot
// 64 i + col, col = i ^ c for mask c), output to the slot's P and E.
template <int N, class AR, int MODE = kWhole>
__device__ __forceinline__ void stage1_warp(uint32_t tile, uint32_t lane, uint32_t o, char* P, uint32_t* Eslot,
                                            TiledCtrl* ws, int s, int gen, uint32_t R, uint64_t pol_keep,
                                            uint32_t k = 0u) {
  using GE = Geo<N, kScratchEntry<AR>>;
  constexpr uint32_t ES = sizeof(typename AR::Raw);
  using SB = S1Bits<ES>;
  const uint32_t c8 = lane & 7u, la = lane >> 3;
  const uint32_t c = (o << 3) | c8;
  const uint32_t ua = ((la & 1u) << SB::A0) | ((la >> 1) << SB::A1);  // lane part of the phase-A index
  const uint32_t ub = ((la & 1u) << SB::B0) | ((la >> 1) << SB::B1);  // lane part of the phase-B index
  auto slot = [&](uint32_t v) { return (v << 6) | (v ^ c); };
  const uint32_t sa = slot(ua), xa = slot(SB::xrow(ua)), xb = slot(SB::xrow(ub));
  typename AR::Raw raw[16];
  uint32_t emax = 0;
  // upper-triangle mode: a tile below the diagonal holds the mirror tile, whose element (col, v)
  // is the conjugate of (v, col); in a diagonal tile (k = 0) the entries below its diagonal are
  // read the same way from the tile itself, and the diagonal's imaginary parts are dropped.
  // slot of (col, v) = slot of (v, col) ^ c ^ (c << 6), col = v ^ c
  // A mirror read's bank group is set by the row v alone, which a quarter-warp's lanes share, so
  // on a tile below the diagonal lane c8 reads its rows in the order v ^ c8 (register j holds row
  // ua ^ reg_a(j) ^ c8, with reg_a(t) = t for t < 8 in both bit assignments): the 8 (16-byte
  // elements) or 16 (8-byte) lanes of one wavefront then hit distinct banks. A register
  // transform of inputs permuted by XOR with t is the transform times (-1)^popc(k & t) at output
  // k, undone after wht_regs by exact negations.
  const bool below = MODE == kUpper && ((R << kTB) ^ (k << kCB)) < (R << kTB);
  const bool diag = MODE == kUpper && k == 0u;
  const uint32_t hc = c ? 31u - (uint32_t)__clz(c) : 32u;  // top set bit of the mask (diagonal tiles)
  const uint32_t rot = below ? c8 : 0u;
  const uint32_t sbase = below ? sa ^ sreg(rot) ^ c ^ (c << 6) : sa;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const uint32_t v = ua ^ reg_a<SB>(j) ^ rot;
    const bool mirror = below || (diag && hc < 32u && ((v >> hc) & 1u));  // element (v, v ^ c) lies below
    const uint32_t a = tile + ((sbase ^ sreg(reg_a<SB>(j))) ^ (!below && mirror ? c | (c << 6) : 0u)) * ES;
    if constexpr (ES == 16) {
      raw[j] = AR::raw_unpack(lds128(a));
    } else {
      const uint2 q = lds64(a);
      raw[j] = AR::raw_unpack(make_uint4(q.x, q.y, 0u, 0u));
    }
    if (MODE == kUpper) {
      if (mirror) raw[j] = AR::conj(raw[j]);
      if (diag && c == 0u) raw[j] = AR::real_part(raw[j]);
    }
    emax = max(emax, AR::exp_key(raw[j]));
  }
  uint32_t Ekey = 0;
  if constexpr (AR::kScaled) {
    emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, 8));
    emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, 16));
    Ekey = emax;
  }
  const typename AR::Conv cv = AR::make_conv(N, Ekey, 0);
  typename AR::Elem v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = AR::template convert<0>(raw[j], cv, 0u);
  wht_regs<AR, 4, 16>(v);
  if constexpr (MODE == kUpper) {
    if (below) {
      const uint32_t m0 = 0u - (rot & 1u), m1 = 0u - ((rot >> 1) & 1u), m2 = 0u - ((rot >> 2) & 1u);
#pragma unroll
      for (int j = 1; j < 16; ++j)
        if (j & 7) negate_where(v[j], ((j & 1) ? m0 : 0u) ^ ((j & 2) ? m1 : 0u) ^ ((j & 4) ? m2 : 0u));
    }
  }
  // exchange within the warp's own slots (the octet's 8 slots of each row): element u goes to
  // the slot of row xrow(u), written in phase A's layout and read in phase B's
  __syncwarp();  // every lane's tile reads are done
  if constexpr (ES == 16) {
#pragma unroll
    for (int j = 0; j < 16; ++j) sts128(tile + (xa ^ sreg(SB::xrow(reg_a<SB>(j)))) * 16u, AR::pack(v[j]));
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = AR::unpack(lds128(tile + (xb ^ sreg(SB::xrow(reg_b<SB>(j)))) * 16u));
  } else {  // 8-byte slots: the first and the second halves of the values in two rounds
    uint2 h[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint4 q = AR::pack(v[j]);
      sts64(tile + (xa ^ sreg(SB::xrow(reg_a<SB>(j)))) * 8u, q.x, q.y);
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 16; ++j) h[j] = lds64(tile + (xb ^ sreg(SB::xrow(reg_b<SB>(j)))) * 8u);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint4 q = AR::pack(v[j]);
      sts64(tile + (xa ^ sreg(SB::xrow(reg_a<SB>(j)))) * 8u, q.z, q.w);
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint2 q = lds64(tile + (xb ^ sreg(SB::xrow(reg_b<SB>(j)))) * 8u);
      v[j] = AR::unpack(make_uint4(h[j].x, h[j].y, q.x, q.y));
    }
  }
  wht_regs<AR, 2, 16>(v);  // register bits 0, 1 hold row bits A0, A1
  // P[chunk][R][t]: chunk = 8o... + (w >> LTPW), t = (w mod TPW) << 3 | c8
  const uint32_t pe = o * (uint32_t)(GE::NCH * GE::NR * GE::TPI) + R * (uint32_t)GE::TPI + c8 + s1_w_off<N>(ub);
  if constexpr (kScratchEntry<AR> == 16) {
    uint4* Pp = reinterpret_cast<uint4*>(P) + pe;
#pragma unroll
    for (int j = 0; j < 16; ++j) st_hint(Pp + s1_w_off<N>(reg_b<SB>(j)), AR::pack(v[j]), pol_keep);
  } else {
    uint2* Pp = reinterpret_cast<uint2*>(P) + pe;
#pragma unroll
    for (int j = 0; j < 16; ++j) st_hint(Pp + s1_w_off<N>(reg_b<SB>(j)), AR::pack_rounded(v[j]), pol_keep);
  }
  if (la == 0u) {
    Eslot[(o * (uint32_t)GE::NR + R) * 8u + c8] = Ekey;
    if constexpr (AR::kScaled) red_max(&ws->emax[s][c], ((uint32_t)(gen + 1) << 11) | key_exp<AR>(Ekey));
  }
}

// ---------------------------------------------------------------------- stage 2 --
// Register part of the output index h at stage 2's second phase (register bit k): the tile
// bits below RLB, then the top bits of h that stay in registers.
template <int N>
__host__ __device__ constexpr int s2_hpos(int k) {
  using GE = Geo<N>;
  return k < GE::RLB ? k : k + (5 - GE::LTPW);
}
template <int N>
__host__ __device__ constexpr uint32_t s2_hreg(int j) {
  uint32_t h = 0;
  for (int k = 0; k < 4; ++k)
    if ((j >> k) & 1) h |= 1u << s2_hpos<N>(k);
  return h;
}

// Warp p of stage-2 item jj of block k: transforms p TPW .. p TPW + TPW - 1 of the chunk, held
// at `region` as [R][TPW] scratch entries; Es = E[R][c8] of the chunk's octet, emax8 = the
// octet's tagged class maxima. The exchange runs on 16-byte entries: in `region` itself (16-byte
// scratch entries), or (8-byte entries: `region` holds 4 KiB) entries 0..255 in `region` and
// 256..511 in `twin`, this warp's 4 KiB in the upper half of the chunk area.
template <int N, class AR, int MODE = 0>
__device__ __forceinline__ void stage2_warp(uint32_t region, uint32_t twin, uint32_t Es, uint32_t emax8, uint32_t lane,
                                            uint32_t p, uint32_t k, uint32_t jj, void* __restrict__ out,
                                            unsigned long long obase, uint64_t pol_out, ShardArgs sa = ShardArgs{N, 0u}) {
  constexpr int SE = kScratchEntry<AR>;
  using GE = Geo<N, SE>;
  constexpr int RLB = GE::RLB, LTPW = GE::LTPW;
  constexpr uint32_t TPW = GE::TPW;
  constexpr uint32_t GM = 8u / TPW - 1u;  // tile bits that select the bank group
  const uint32_t tt = lane & (TPW - 1u), rl = lane >> LTPW;
  const uint32_t t = p * TPW + tt, c8 = t & 7u, wlo = t >> 3;
  const uint32_t o = jj / GE::NCH, whi = jj % GE::NCH;
  const uint32_t w = (whi << LTPW) | wlo;
  const uint32_t x = ((MODE == kShard) ? sa.xhi : 0u) | (k << kCB) | (o << 3) | c8;
  auto xaddr = [&](uint32_t e) {  // exchange entry e < 512
    if constexpr (SE == 16) return region + e * 16u;
    else return ((e & 256u) ? twin : region) + (e & 255u) * 16u;
  };
  typename AR::Elem v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const uint32_t R = ((uint32_t)j << RLB) | rl;
    if constexpr (SE == 16) {
      v[j] = AR::unpack(lds128(region + (R * TPW + tt) * 16u));
    } else {
      v[j] = AR::unpack_rounded(lds64(region + (R * TPW + tt) * 8u));
    }
  }
  typename AR::Conv cv;
  if constexpr (kRegrid<AR>) {
    cv = AR::make_conv(N, exp_to_key<AR>(lds32(emax8 + 4u * c8) & 0x7FFu), -N);
#pragma unroll
    for (int j = 0; j < 16; ++j) AR::regrid(v[j], cv);
  } else if constexpr (AR::kScaled) {
    const int em = (int)(lds32(emax8 + 4u * c8) & 0x7FFu);
    cv = AR::make_conv(N, (uint32_t)em << 20, -N);
    if (!cv.nan) {
      // tile R was converted at scale 2^(s + em - et): shift right by em - et (all-zero tiles
      // have et = 0 and hold zeros)
      const uint32_t e0 = Es + 4u * ((rl * 8u) + c8);  // E[R][c8] of register 0; register j adds 2^RLB j rows
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int et = (int)(lds32(e0 + 4u * 8u * ((uint32_t)j << RLB)) >> 20);
        AR::align(v[j], min(em - et, 63));
      }
    }
  } else {
    cv = AR::make_conv(N, 0u, -N);
  }
  wht_regs<AR, 4, 16>(v);  // the four tile bits above RLB
  if constexpr (SE == 8) __syncwarp();  // every lane's 8-byte reads are done before the region is reused
  // in-place exchange, entry (R, tt) at R' TPW + tt with R' = R_hi . (R_lo ^ (R_hi & GM))
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const uint32_t Rs = ((uint32_t)j << RLB) | (rl ^ ((uint32_t)j & GM));
    sts128(xaddr(Rs * TPW + tt), AR::pack(v[j]));
  }
  __syncwarp();
  const uint32_t hh = rl;  // the same lane bits now hold the low tile bits above RLB
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const uint32_t Rl = (uint32_t)j & ((1u << RLB) - 1u);
    const uint32_t Rh = hh | (((uint32_t)j >> RLB) << (5 - LTPW));
    const uint32_t Rs = (Rh << RLB) | (Rl ^ (Rh & GM));
    v[j] = AR::unpack(lds128(xaddr(Rs * TPW + tt)));
  }
  wht_regs<AR, RLB, 16>(v);
  // c(x, z), z = (h << 6) | w with h = (hh << RLB) | (register part)
  const uint32_t zl = ((hh << RLB) << kCB) | w;
  Addr<N, false> ao;
  ao.init(obase, x, zl);
  constexpr int q0 = s2_hpos<N>(0) + kCB, q1 = s2_hpos<N>(1) + kCB, q2 = s2_hpos<N>(2) + kCB,
                q3 = s2_hpos<N>(3) + kCB;
  BitSum<q0, q1, q2, q3> xo;
  xo.init(x);
  const uint32_t ko = (uint32_t)__popc(x & zl);
  if constexpr (MODE == kShard) {
    // compact index of the shard's output: n's low 2m bits, then the top z bits
    const uint32_t lomask = (uint32_t)((1ull << (2 * sa.m)) - 1ull);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t z = zl | (s2_hreg<N>(j) << kCB);
      const uint32_t n = (uint32_t)(ao.at(s2_hreg<N>(j) << kCB) - obase);
      const unsigned long long idx = obase + ((n & lomask) | ((z >> sa.m) << (2 * sa.m)));
      AR::store_hint(out, idx, v[j], cv, ko + xo.at(j), pol_out);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) AR::store_hint(out, ao.at(s2_hreg<N>(j) << kCB), v[j], cv, ko + xo.at(j), pol_out);
  }
}

// ---------------------------------------------------------------------- consumers --
template <int N, class AR, int MODE>
__device__ void consumer(void* __restrict__ out, int count, TiledCtrl* ws, Shared& sh, uint32_t buf0,
                         uint32_t warp, uint32_t lane, ShardArgs sa) {
  using GE = Geo<N, kScratchEntry<AR>>;
  constexpr uint32_t D = 1u << N;
  const int nbl = (MODE == kShard) ? sa.m - kCB : N - kCB, nb = 1 << nbl;  // mask blocks per matrix (or shard)
  const uint32_t team = warp / kTeamWarps, p = warp % kTeamWarps;
  const int blocks = nb * count;
  const uint64_t pol_keep = policy_evict_last(), pol_first = policy_evict_first();
  char* const P0 = reinterpret_cast<char*>(ws) + GE::kPBase;
  uint32_t* const E0 = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(ws) + GE::kEBase);
  const volatile int* item_of = sh.item;
  for (int use = (int)team;; use += kTeams) {
    const int buf = use % kBufs;
    // The buffer's previous use (use - 3, the other team's) may still be in flight when this
    // team gets here: its phase has the other parity, so a completed parity wait alone could be
    // that older phase. The use tag, written before the producer's arrival, tells them apart.
    const uint32_t full = smem_addr(&sh.full[buf]);
    if (!wait_use(full, (use / kBufs) & 1, &sh.use_of[buf], use, &ws->status)) break;
    if (p == 0 && lane == 0) sh.waited_use[buf] = use;
    const int item = item_of[buf];
    if (item < 0) {
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_addr(&sh.done[use % kRel]));  // lets the release warp see the end
      break;
    }
    Item<N> it;
    it.decode(item, blocks);
    const int s = it.b % GE::NS, gen = it.b / GE::NS;
    const uint32_t addr = buf0 + (uint32_t)(buf * GE::kBuf);
    if (it.s1) {
      stage1_warp<N, AR, MODE>(addr, lane, p, P0 + (size_t)s * GE::kSlotP, E0 + (size_t)s * (GE::kSlotE / 4), ws, s,
                               gen, (uint32_t)it.j, pol_keep, (uint32_t)(it.b & (nb - 1)));
    } else {
      // the slot's data of this item is in shared memory: a relaxed count suffices
      if (p == 0 && lane == 0) red_relaxed_add(&ws->s2_done[s], 1);
      stage2_warp<N, AR, MODE>(addr + p * GE::kSlice, addr + (uint32_t)(GE::kChunkArea / 2) + p * GE::kSlice,
                                addr + (uint32_t)GE::kChunkArea, addr + (uint32_t)(GE::kChunkArea + GE::kEOct), lane, p,
                                (uint32_t)(it.b & (nb - 1)),
                                (uint32_t)it.j, out, (unsigned long long)(it.b >> nbl) * D * ((MODE == kShard) ? 1ull << sa.m : D),
                                pol_first, sa);
    }
    // the warp is done with the buffer (measured faster than handing it back right after its
    // last shared-memory access) and has issued its stores
    fence_proxy_async_shared();  // this lane's generic accesses before the next copy's async writes
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(smem_addr(&sh.empty[buf]));
      mbar_arrive(smem_addr(&sh.done[use % kRel]));
    }
  }
}

template <int N, class AR, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
    twostage_kernel(const __grid_constant__ CUtensorMap gmap, const __grid_constant__ CUtensorMap smap,
                    void* __restrict__ out, int count, TiledCtrl* ws, ShardArgs sa) {
  extern __shared__ __align__(1024) char bufs[];
  __shared__ Shared sh;
  const uint32_t t = threadIdx.x, warp = t >> 5, lane = t & 31u;
  const uint32_t buf0 = smem_addr(bufs);
  if (t == 0) {
    for (int q = 0; q < kRel; ++q) mbar_init(smem_addr(&sh.done[q]), kTeamWarps);
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(smem_addr(&sh.full[b]), 1);
      mbar_init(smem_addr(&sh.empty[b]), kTeamWarps);
      sh.waited_use[b] = -1;
      sh.issued_use[b] = -1;
      sh.use_of[b] = -1;
    }
    sh.released = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp < (uint32_t)kConsumerWarps) {
    regs_inc<kConsumerRegs>();
    consumer<N, AR, MODE>(out, count, ws, sh, buf0, warp, lane, sa);
  } else {
    regs_dec<kHelperRegs>();
    if (warp == (uint32_t)kConsumerWarps && lane == 0) producer<N, AR, MODE>(&gmap, &smap, count, ws, sh, buf0, sa);
    if (warp == (uint32_t)kConsumerWarps + 1 && lane == 0) releaser(ws, sh);
  }
  __syncwarp();
  __syncthreads();
  // after a wait gave up: wait (bounded) for copies still landing in buffers nobody waited for
  if (t == 0) {
    for (int b = 0; b < kBufs; ++b) {
      const int u = sh.issued_use[b];
      if (u <= sh.waited_use[b]) continue;
      wait_use(smem_addr(&sh.full[b]), (u / kBufs) & 1, &sh.use_of[b], u, &ws->status);
    }
  }
}

// MODE kShard: G is the block-XOR layout of shard sa (one matrix, count = 1); else sa = {N, 0}.
// MODE kUpper: G is Hermitian and read from its upper triangle.
template <int N, class AR, int MODE = 0>
cudaError_t launch_t(const void* G, int count, void* out, cudaStream_t st, ShardArgs sa = ShardArgs{N, 0u}) {
  using GE = Geo<N, kScratchEntry<AR>>;
  void* ws = nullptr;
  cudaError_t e = tiled_workspace(st, GE::kWorkspace, &ws);
  if (e != cudaSuccess) return e;
  CUtensorMap gmap, smap;
  e = (MODE == kShard) ? tiled_tensor_map_rows(&gmap, G, sa.m, (1ll << N) * count, (int)sizeof(typename AR::Raw))
            : tiled_tensor_map(&gmap, G, N, count, (int)sizeof(typename AR::Raw));
  if (e != cudaSuccess) return e;
  // a warp's slice of one tile row: TPW entries in 8-byte words
  e = scratch_tensor_map4(&smap, reinterpret_cast<char*>(ws) + GE::kPBase, GE::NS * GE::NR, GE::NR,
                          GE::TPW * kScratchEntry<AR> / 8);
  if (e != cudaSuccess) return e;
  auto kern = twostage_kernel<N, AR, MODE>;
  constexpr size_t smem = kBufs * GE::kBuf;
  static int grid = 0;  // one CTA per SM
  if (!grid) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
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
  kern<<<grid, kThreads, smem, st>>>(gmap, smap, out, count, reinterpret_cast<TiledCtrl*>(ws), sa);
  return cudaGetLastError();
}

template <class AR>
cudaError_t launch_n(const void* G, int N, int count, void* out, cudaStream_t st) {
  switch (N) {
    case 12: return launch_t<12, AR>(G, count, out, st);
    case 13: return launch_t<13, AR>(G, count, out, st);
    case 14: return launch_t<14, AR>(G, count, out, st);
    default: return cudaErrorNotSupported;
  }
}

// Hermitian G read from its upper triangle (real outputs: AR is a ReOut policy).
template <class AR>
cudaError_t launch_upper_n(const void* G, int N, int count, void* out, cudaStream_t st) {
  switch (N) {
    case 12: return launch_t<12, AR, kUpper>(G, count, out, st);
    case 13: return launch_t<13, AR, kUpper>(G, count, out, st);
    case 14: return launch_t<14, AR, kUpper>(G, count, out, st);
    default: return cudaErrorNotSupported;
  }
}

// x-class shard x_hi of 2^k from its block-XOR layout L (needs N - k >= 6).
template <class AR>
cudaError_t launch_xhi_n(const void* L, int N, int k, uint32_t x_hi, void* out, cudaStream_t st) {
  const ShardArgs sa{N - k, x_hi << (N - k)};
  if (N - k < kCB) return cudaErrorNotSupported;
  switch (N) {
    case 12: return launch_t<12, AR, kShard>(L, 1, out, st, sa);
    case 13: return launch_t<13, AR, kShard>(L, 1, out, st, sa);
    case 14: return launch_t<14, AR, kShard>(L, 1, out, st, sa);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace
}  // namespace ts
}  // namespace pauli

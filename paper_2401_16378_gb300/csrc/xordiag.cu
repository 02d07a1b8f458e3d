// xordiag.cu -- XOR-diagonal gather + Walsh-Hadamard transform (decompose and compose).
//
// For an XY-mask x (Eq. (11)) every coefficient with that mask reads the same 2^N matrix
// elements: the XOR-diagonal e_x[r] = G[r, r ^ x]. With the lambda of Eq. (12) written as
// (-i)^popc(x&z) (-1)^popc(i&z), Eq. (13) for all z at once is
//   c(x, z) = 2^-N * i^popc(x&z) * W_x[z],   W_x[z] = sum_r (-1)^popc(r&z) e_x[r],
// a length-2^N Walsh-Hadamard transform (WHT) over r, followed by an exact phase and scale.
// That is O(N 2^N) per x instead of O(4^N), and the whole decomposition reads G once and
// writes the 4^N coefficients once. Composition (Eq. (1)) is the inverse map:
//   G[r, r ^ x] = sum_z (-1)^popc(r&z) (-i)^popc(x&z) c(x, z).
//
// Work unit: 8192 elements, 16 per thread of a 512-thread CTA, held in registers. For
// N <= 12 a unit is 2^K consecutive XY-masks (the "classes", K = 13 - N) times all 2^N rows,
// in one CTA. Consecutive x share DRAM sectors (G[r, r^x] and G[r, r^x^1] are adjacent),
// and their coefficients n(x, z), n(x^1, z) are adjacent too, so a unit reads and writes
// whole sectors. For N >= 13 a unit is one class pair (x, x^1) over all rows, shared by a
// cluster of 2^(N-12) CTAs (see xordiag_cluster_kernel).
// The transform runs in register phases of up to 4 butterfly stages, with the data
// re-distributed between threads through shared memory (XOR-swizzled 16-byte slots).
// The kernels are persistent: each CTA (or cluster) walks a strided list of units and,
// while it computes one, prefetches the rows of its next unit into L2, so HBM stays busy
// during the arithmetic and the stores of one unit drain while the next one computes.
//
// Arithmetic:
//  complex128: every class is converted to int64 fixed point with a per-class power-of-two
//    scale (block floating point), chosen from the class's largest exponent so that 2^N
//    terms cannot overflow; the transform is then exact (integer adds), and the only
//    roundings are the input quantisation (truncation, < 2^(N-61) max|G| per coefficient)
//    and the final truncating conversion back to FP64 (< 1 ulp). No FP64 instruction is
//    used: on GB300 the FP64 pipe issues ~2 ops/clk/SM while the integer pipes issue ~128.
//  complex64: TwoSum-compensated FP32: each value is an unevaluated pair (hi, lo); every
//    butterfly adds with TwoSum and carries the exact rounding error into lo.
#include "kernels.h"
#include "xordiag_impl.cuh"

namespace pauli {
namespace {
using namespace xd;

// ----------------------------------------------------------------- single-CTA units --
// A unit = 2^K classes x 2^N rows in one CTA (N <= UB - 1). One unit per CTA, in blockIdx
// order: neighbouring units share DRAM lines (a 128-byte line holds 8 consecutive
// classes of a row), and CTAs launched together keep those shared lines in L2 until all of
// them have read it. Each CTA prefetches into L2 the unit one resident wave ahead -- the unit
// that will run on an SM after this wave -- so HBM stays busy while this one computes.
template <int UB, int N, class AR, bool COMPOSE>
__global__ void __launch_bounds__(Unit<UB>::kThreads, Unit<UB>::kMinBlocks)
    xordiag_kernel(const void* __restrict__ in, void* __restrict__ out, int scale_exp, unsigned long long units,
                   unsigned long long ahead) {
  using LY = Layout<UB, N>;
  constexpr int K = LY::K;
  constexpr uint32_t D = 1u << N;
  extern __shared__ __align__(16) uint4 xbuf[];
  __shared__ uint32_t smax[1 << K];
  const uint32_t t = threadIdx.x;
  const uint32_t xaddr = (uint32_t)__cvta_generic_to_shared(xbuf);
  const unsigned long long units_per_mat = D >> K;
  const unsigned long long unit = blockIdx.x;
  const unsigned long long nu = unit + ahead;
  auto prefetch_ahead = [&]() {
    if (nu < units)
      unit_prefetch<UB, N, AR, COMPOSE>(in, (nu / units_per_mat) * (unsigned long long)D * D,
                                        (uint32_t)(nu % units_per_mat) << K, t);
  };
  run_unit<UB, N, AR, COMPOSE>(in, out, (unit / units_per_mat) * (unsigned long long)D * D,
                               (uint32_t)(unit % units_per_mat) << K, scale_exp, xaddr, smax, t, prefetch_ahead);
}

// ------------------------------------------------------------------------- CTA clusters --
// A class pair (x, x^1) of 2^(N+1) elements larger than one unit is shared by a cluster of
// CL = 2^(N-LB) CTAs, LB = UB - 1: CTA q owns the rows (decompose) or YZ-masks (compose)
// whose top N-LB bits equal q, transforms their LB low bits locally exactly as the
// single-CTA kernel does, and the remaining N-LB butterfly stages combine the CL partial
// transforms through distributed shared memory: after a cluster barrier, CTA q' reads from
// every CTA of the cluster the partial results for its slice of the LB low output bits (the
// slice whose top log2(CL) bits equal q') and finishes the CL-point transform in registers.
// The fixed-point scale of each class is the cluster-wide maximum exponent.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t map_shared_u32(uint32_t local, uint32_t rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(local), "r"(rank));
  return out;
}
__device__ __forceinline__ uint4 ld_dsmem16(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared::cluster.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_dsmem_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

template <int UB, int N, class AR, bool COMPOSE>
__global__ void __launch_bounds__(Unit<UB>::kThreads, Unit<UB>::kMinBlocks)
    xordiag_cluster_kernel(const void* __restrict__ in, void* __restrict__ out, int scale_exp,
                           unsigned long long units, unsigned long long ahead) {
  constexpr int LB = UB - 1;  // local row bits (1 class bit)
  using LY = Layout<UB, LB>;
  constexpr int CLB = N - LB;
  constexpr uint32_t CL = 1u << CLB;
  constexpr uint32_t D = 1u << N;
  constexpr int WB = UB - 9;     // warp-index bits
  constexpr int POSB = 4 - CLB;  // log2 of output positions per thread in the combine
  static_assert(CLB >= 1 && CLB <= 3, "cluster of 2, 4 or 8 CTAs");
  extern __shared__ __align__(16) uint4 xbuf[];
  __shared__ uint32_t smax[2];

  const uint32_t t = threadIdx.x;
  const uint32_t xaddr = (uint32_t)__cvta_generic_to_shared(xbuf);
  const uint32_t q = cluster_rank();
  const unsigned long long units_per_mat = D >> 1;
  const uint32_t y0 = (q << LB) | (LY::thread_u(0, t) >> 1);
  const int out_scale = COMPOSE ? scale_exp : -N;
  // combine mapping: lane bits (class, y0..y3), warp bits y4.., POSB position bits, rank bits on top
  const uint32_t lane_part = ((t >> 1) & 15u) | ((t >> 5) << 4);
  uint32_t peer_x[CL], peer_m[CL];
#pragma unroll
  for (uint32_t r = 0; r < CL; ++r) {
    peer_x[r] = map_shared_u32(xaddr, r);
    peer_m[r] = map_shared_u32((uint32_t)__cvta_generic_to_shared(&smax[t & 1u]), r);
  }

  {
    const unsigned long long unit = blockIdx.x >> CLB;  // one class pair per cluster
    const unsigned long long kmat = unit / units_per_mat;
    const uint32_t x = ((uint32_t)(unit % units_per_mat) << 1) | (t & 1u);
    const unsigned long long base = kmat * (unsigned long long)D * D;
    Addr<N, !COMPOSE> ain;
    ain.init(base, x, y0);
    typename AR::Raw raw[16];
    uint32_t emax = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      raw[j] = AR::load(in, ain.at(LY::reg_u(0, j) >> 1));
      emax = max(emax, AR::exp_key(raw[j]));
    }
    {
      const unsigned long long nu = unit + ahead;
      if (nu < units) {
        Addr<N, !COMPOSE> an;
        an.init((nu / units_per_mat) * (unsigned long long)D * D, ((uint32_t)(nu % units_per_mat) << 1) | (t & 1u),
                y0);
#pragma unroll
        for (int j = 0; j < 16; ++j) AR::prefetch(in, an.at(LY::reg_u(0, j) >> 1));
      }
    }
    uint32_t Ekey = 0;
    if constexpr (AR::kScaled) {
      if (t < 2) smax[t] = 0;
      __syncthreads();
#pragma unroll
      for (int m = 2; m < 32; m <<= 1) emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, m));
      if ((t & 31u) < 2) atomicMax(&smax[t & 1u], emax);
      cluster_sync_all();  // every CTA's smax is final
#pragma unroll
      for (uint32_t r = 0; r < CL; ++r) Ekey = max(Ekey, ld_dsmem_u32(peer_m[r]));
    }
    const typename AR::Conv cv = AR::make_conv(N, Ekey, out_scale);
    typename AR::Elem v[16];
    {
      const uint32_t kt = COMPOSE ? 3u * (uint32_t)__popc(x & y0) : 0u;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const uint32_t k = COMPOSE ? kt + 3u * (uint32_t)__popc(x & (LY::reg_u(0, j) >> 1)) : 0u;
        v[j] = AR::template convert<0>(raw[j], cv, k);
      }
    }
    wht_regs<AR, LY::gcount(0)>(v);
    exchange<LY, AR, 0>(v, xaddr, t);
    wht_regs<AR, LY::gcount(1)>(v);
    exchange<LY, AR, 1>(v, xaddr, t);
    wht_regs<AR, LY::gcount(2)>(v);
    // publish the local transform
    __syncthreads();
    {
      const uint32_t ut = LY::thread_u(2, t);
      const uint32_t ft = ut ^ swz_term(ut);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        sts128(xaddr + 16u * (ft ^ (LY::reg_u(2, j) ^ swz_term(LY::reg_u(2, j)))), AR::pack(v[j]));
    }
    cluster_sync_all();
#pragma unroll
    for (int p = 0; p < (1 << POSB); ++p) {
      const uint32_t ylow = lane_part | ((uint32_t)p << (4 + WB)) | (q << (LB - CLB));  // low LB output bits
      const uint32_t u = (t & 1u) | (ylow << 1);
      const uint32_t off = 16u * (u ^ swz_term(u));
      typename AR::Elem w[CL];
#pragma unroll
      for (uint32_t r = 0; r < CL; ++r) w[r] = AR::unpack(ld_dsmem16(peer_x[r] + off));
#pragma unroll
      for (int b = 0; b < CLB; ++b)
#pragma unroll
        for (uint32_t r = 0; r < CL; ++r)
          if (!((r >> b) & 1u)) AR::bfly(w[r], w[r | (1u << b)]);
      Addr<N, COMPOSE> ao;
      ao.init(base, x, ylow);
      const uint32_t kt = COMPOSE ? 0u : (uint32_t)__popc(x & ylow);
#pragma unroll
      for (uint32_t r = 0; r < CL; ++r) {
        const uint32_t yj = r << LB;  // top output bits
        const uint32_t k = COMPOSE ? 0u : kt + (uint32_t)__popc(x & yj);
        AR::store(out, ao.at(yj), w[r], cv, k);
      }
    }
    cluster_sync_all();  // peers may still be reading this CTA's shared memory
  }
}

// ------------------------------------------------------------------------------- launch --
int device_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

template <int UB, int N, class AR, bool COMPOSE>
cudaError_t launch_one(const void* in, long long count, int scale_exp, void* out, cudaStream_t st) {
  constexpr size_t smem = Unit<UB>::kSmem;
  auto kern = xordiag_kernel<UB, N, AR, COMPOSE>;
  static int resident = 0;  // CTAs per SM (one device per process in this library)
  if (!resident) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, Unit<UB>::kThreads, smem);
    if (e != cudaSuccess) return e;
    resident = n > 0 ? n : 1;
  }
  const unsigned long long units = (unsigned long long)count * ((1ull << (2 * N)) >> UB);
  if (units > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
  const unsigned long long ahead = (unsigned long long)device_sms() * resident;
  kern<<<(unsigned)units, Unit<UB>::kThreads, smem, st>>>(in, out, scale_exp, units, ahead);
  return cudaGetLastError();
}

template <int UB, int N, class AR, bool COMPOSE>
cudaError_t launch_cluster(const void* in, long long count, int scale_exp, void* out, cudaStream_t st) {
  constexpr size_t smem = Unit<UB>::kSmem;
  constexpr unsigned CL = 1u << (N - (UB - 1));
  auto kern = xordiag_cluster_kernel<UB, N, AR, COMPOSE>;
  static int max_clusters = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(Unit<UB>::kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (!max_clusters) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cfg.gridDim = dim3(CL * 1024);
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) return e;
    max_clusters = n > 0 ? n : 1;
  }
  const unsigned long long units = (unsigned long long)count * ((1ull << N) >> 1);
  if (units * CL > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
  cfg.gridDim = dim3((unsigned)(units * CL));
  return cudaLaunchKernelEx(&cfg, kern, in, out, scale_exp, units, (unsigned long long)max_clusters);
}

// Unit size 2^13: N in [7, 12] single CTA, [13, 15] clusters of 2..8.
template <class AR, bool COMPOSE>
cudaError_t dispatch_u13(int N, const void* in, long long count, int scale_exp, void* out, cudaStream_t st) {
  switch (N) {
    case 7: return launch_one<13, 7, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 8: return launch_one<13, 8, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 9: return launch_one<13, 9, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 10: return launch_one<13, 10, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 11: return launch_one<13, 11, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 12: return launch_one<13, 12, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 13: return launch_cluster<13, 13, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 14: return launch_cluster<13, 14, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 15: return launch_cluster<13, 15, AR, COMPOSE>(in, count, scale_exp, out, st);
    default: return cudaErrorNotSupported;
  }
}
// Unit size 2^12: N in [6, 11] single CTA, [12, 14] clusters of 2..8.
template <class AR, bool COMPOSE>
cudaError_t dispatch_u12(int N, const void* in, long long count, int scale_exp, void* out, cudaStream_t st) {
  switch (N) {
    case 6: return launch_one<12, 6, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 7: return launch_one<12, 7, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 8: return launch_one<12, 8, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 9: return launch_one<12, 9, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 10: return launch_one<12, 10, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 11: return launch_one<12, 11, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 12: return launch_cluster<12, 12, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 13: return launch_cluster<12, 13, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 14: return launch_cluster<12, 14, AR, COMPOSE>(in, count, scale_exp, out, st);
    default: return cudaErrorNotSupported;
  }
}

bool variant_has(int variant, int N) {
  if (variant == kVariantUnit13) return N >= 7 && N <= 15;
  if (variant == kVariantUnit12) return N >= 6 && N <= 14;
  return false;
}

// Chosen variant per (N, dtype, direction): 0 = built-in default. Set by the autotuner.
int g_variant[2][2][17];

int default_variant(int N) { return N >= 7 ? kVariantUnit13 : kVariantUnit12; }

}  // namespace

bool xordiag_supported(int N) { return N >= 6 && N <= 15; }

bool xordiag_variant_supported(int variant, int N) { return variant_has(variant, N); }

int xordiag_get_variant(int N, bool c64, bool compose) {
  if (N < 0 || N > 16) return 0;
  const int v = g_variant[c64][compose][N];
  return v ? v : (xordiag_supported(N) ? default_variant(N) : 0);
}

void xordiag_set_variant(int N, bool c64, bool compose, int variant) {
  if (N >= 0 && N <= 16) g_variant[c64][compose][N] = variant;
}

cudaError_t launch_xordiag(const void* in, int N, long long count, bool c64, bool compose, int scale_exp, void* out,
                           cudaStream_t s, int variant) {
  if (!variant) variant = xordiag_get_variant(N, c64, compose);
  if (!variant_has(variant, N)) return cudaErrorNotSupported;
  if (variant == kVariantUnit12) {
    if (c64)
      return compose ? dispatch_u12<ArC64, true>(N, in, count, scale_exp, out, s)
                     : dispatch_u12<ArC64, false>(N, in, count, scale_exp, out, s);
    return compose ? dispatch_u12<ArC128, true>(N, in, count, scale_exp, out, s)
                   : dispatch_u12<ArC128, false>(N, in, count, scale_exp, out, s);
  }
  if (c64)
    return compose ? dispatch_u13<ArC64, true>(N, in, count, scale_exp, out, s)
                   : dispatch_u13<ArC64, false>(N, in, count, scale_exp, out, s);
  return compose ? dispatch_u13<ArC128, true>(N, in, count, scale_exp, out, s)
                 : dispatch_u13<ArC128, false>(N, in, count, scale_exp, out, s);
}

}  // namespace pauli

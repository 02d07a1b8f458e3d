// xordiag_kernels.cuh -- kernels, launchers and per-shape dispatch of the XOR-diagonal path
// (included by the per-dtype translation units xordiag_*.cu).
#pragma once
#include <type_traits>

#include "kernels.h"
#include "xordiag_impl.cuh"

namespace pauli {
namespace xk {
using namespace xd;

// ----------------------------------------------------------------- single-CTA units --
// A unit = 2^K classes x 2^N rows in one CTA (N <= UB - 1). One unit per CTA, in blockIdx
// order: neighbouring units share DRAM lines (a 128-byte line holds 8 consecutive classes of
// a row), and CTAs launched together read them close in time. Each CTA prefetches into L2
// the unit one resident wave ahead -- the unit that will run on an SM after this wave.
// EPI: NoEpi, or the fused forms (WeightInEpi for compose; NormOutEpi for decompose, which
// writes the unit's partial loss to ea.partial[unit] in a fixed order).
template <int UB, int RB, int N, class AR, bool COMPOSE, class EPI = NoEpi>
__global__ void __launch_bounds__(Unit<UB, RB>::kThreads, Unit<UB, RB>::kMinBlocks)
    xordiag_kernel(const void* __restrict__ in, void* __restrict__ out, int scale_exp, unsigned long long units,
                   unsigned long long ahead, EpiArgs ea) {
  using LY = Layout<UB, N, RB>;
  constexpr int K = LY::K;
  constexpr uint32_t D = 1u << N;
  extern __shared__ __align__(16) uint4 xbuf[];
  __shared__ uint32_t smax[1 << K];
  const uint32_t t = threadIdx.x;
  const uint32_t xaddr = (uint32_t)__cvta_generic_to_shared(xbuf);
  const unsigned long long units_per_mat = D >> K;
  const unsigned long long unit = blockIdx.x;
  const unsigned long long nu = unit + ahead;
  // The L2 prefetch of the next wave's unit pays where a unit's row segments are short and the
  // CTAs few; measured on GB300 it costs time (issue slots and load-queue entries) for
  // 4096-element units from N = 10 on, for 8192-element decompositions at N = 12 and for
  // complex64 8192-element compositions at N = 12.
  constexpr bool kPrefetch =
      UB == 13 ? (N <= 11 || (COMPOSE && !std::is_same<AR, ArC64>::value)) : N <= 9;
  auto prefetch_ahead = [&]() {
    if (kPrefetch && nu < units)
      unit_prefetch<UB, RB, N, AR, COMPOSE>(in, (nu / units_per_mat) * (unsigned long long)D * D,
                                            (uint32_t)(nu % units_per_mat) << K, t);
  };
  const unsigned long long base = (unit / units_per_mat) * (unsigned long long)D * D;
  const double part = run_unit<UB, RB, N, AR, COMPOSE, decltype(prefetch_ahead), EPI>(
      in, out, base, (uint32_t)(unit % units_per_mat) << K, scale_exp, xaddr, smax, t, prefetch_ahead, ea);
  if constexpr (EPI::kNormOut) {
    // fixed-tree block sum of the threads' shares
    __shared__ double wsum[Unit<UB, RB>::kThreads / 32];
    double v = part;
#pragma unroll
    for (int m = 16; m; m >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
    if ((t & 31u) == 0) wsum[t >> 5] = v;
    __syncthreads();
    if (t == 0) {
      double tot = 0.0;
#pragma unroll
      for (int i = 0; i < Unit<UB, RB>::kThreads / 32; ++i) tot += wsum[i];
      ea.partial[unit] = tot;
    }
  } else {
    (void)part;
  }
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

template <int UB, int RB, int N, class AR, bool COMPOSE>
__global__ void __launch_bounds__(Unit<UB, RB>::kThreads, Unit<UB, RB>::kMinBlocks)
    xordiag_cluster_kernel(const void* __restrict__ in, void* __restrict__ out, int scale_exp,
                           unsigned long long units, unsigned long long ahead) {
  constexpr int LB = UB - 1;  // local row bits (1 class bit)
  using LY = Layout<UB, LB, RB>;
  constexpr int E = LY::E;
  constexpr int LAST = LY::NPH - 1;
  constexpr int CLB = N - LB;
  constexpr uint32_t CL = 1u << CLB;
  constexpr uint32_t D = 1u << N;
  constexpr int WB = UB - RB - 5;  // warp-index bits
  constexpr int POSB = RB - CLB;   // log2 of output positions per thread in the combine
  static_assert(CLB >= 1 && CLB <= 3 && POSB >= 0, "cluster of 2, 4 or 8 CTAs");
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
  const unsigned long long unit = blockIdx.x >> CLB;  // one class pair per cluster
  const unsigned long long kmat = unit / units_per_mat;
  const uint32_t x = ((uint32_t)(unit % units_per_mat) << 1) | (t & 1u);
  const unsigned long long base = kmat * (unsigned long long)D * D;
  Addr<N, !COMPOSE> ain;
  ain.init(base, x, y0);
  typename AR::Raw raw[E];
  uint32_t emax = 0;
#pragma unroll
  for (int j = 0; j < E; ++j) {
    raw[j] = AR::load(in, ain.at(LY::reg_u(0, j) >> 1));
    emax = max(emax, AR::exp_key(raw[j]));
  }
  {
    const unsigned long long nu = unit + ahead;
    if (nu < units) {
      Addr<N, !COMPOSE> an;
      an.init((nu / units_per_mat) * (unsigned long long)D * D, ((uint32_t)(nu % units_per_mat) << 1) | (t & 1u), y0);
#pragma unroll
      for (int j = 0; j < E; ++j) AR::prefetch(in, an.at(LY::reg_u(0, j) >> 1));
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
  BitSum<LB, (CLB > 1 ? LB + 1 : -1), (CLB > 2 ? LB + 2 : -1), -1> xt;
  xt.init(x);
  typename AR::Elem v[E];
  {
    BitSum<LY::regrow(0, 0), LY::regrow(0, 1), LY::regrow(0, 2), LY::regrow(0, 3)> xb;
    xb.init(x);
    const uint32_t kt = COMPOSE ? (uint32_t)__popc(x & y0) : 0u;
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = AR::template convert<0>(raw[j], cv, COMPOSE ? 3u * (kt + xb.at(j)) : 0u);
  }
  local_wht<LY, AR>(v, xaddr, t);
  // publish the local transform
  __syncthreads();
  {
    const uint32_t ut = LY::thread_u(LAST, t);
    const uint32_t ft = ut ^ swz_term(ut);
#pragma unroll
    for (int j = 0; j < E; ++j)
      sts128(xaddr + 16u * (ft ^ (LY::reg_u(LAST, j) ^ swz_term(LY::reg_u(LAST, j)))), AR::pack(v[j]));
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
    for (uint32_t r = 0; r < CL; ++r)  // top output bits r << LB
      AR::store(out, ao.at(r << LB), w[r], cv, COMPOSE ? 0u : kt + xt.at((int)r));
  }
  cluster_sync_all();  // peers may still be reading this CTA's shared memory
}

// ------------------------------------------------------------------------------- launch --
static int device_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

template <int UB, int RB, int N, class AR, bool COMPOSE, class EPI = NoEpi>
cudaError_t launch_one(const void* in, long long count, int scale_exp, void* out, cudaStream_t st,
                       EpiArgs ea = EpiArgs{nullptr, nullptr, nullptr}) {
  constexpr size_t smem = Unit<UB, RB>::kSmem;
  auto kern = xordiag_kernel<UB, RB, N, AR, COMPOSE, EPI>;
  static int resident = 0;  // CTAs per SM (one device per process in this library)
  if (!resident) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, Unit<UB, RB>::kThreads, smem);
    if (e != cudaSuccess) return e;
    resident = n > 0 ? n : 1;
  }
  const unsigned long long units = (unsigned long long)count * ((1ull << (2 * N)) >> UB);
  if (units > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
  const unsigned long long ahead = (unsigned long long)device_sms() * resident;
  kern<<<(unsigned)units, Unit<UB, RB>::kThreads, smem, st>>>(in, out, scale_exp, units, ahead, ea);
  return cudaGetLastError();
}

template <int UB, int RB, int N, class AR, bool COMPOSE>
cudaError_t launch_cluster(const void* in, long long count, int scale_exp, void* out, cudaStream_t st) {
  constexpr size_t smem = Unit<UB, RB>::kSmem;
  constexpr unsigned CL = 1u << (N - (UB - 1));
  auto kern = xordiag_cluster_kernel<UB, RB, N, AR, COMPOSE>;
  static int max_clusters = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(Unit<UB, RB>::kThreads);
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

// Launch shapes: single-CTA units for N in [NMIN, UB - 1], clusters of 2..8 above.
template <int UB, int RB, class AR, bool COMPOSE>
cudaError_t dispatch_shape(int N, const void* in, long long count, int scale_exp, void* out, cudaStream_t st) {
  switch (N) {
    case 6:
      if constexpr (UB == 12) return launch_one<UB, RB, 6, AR, COMPOSE>(in, count, scale_exp, out, st);
      break;
    case 7: return launch_one<UB, RB, 7, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 8: return launch_one<UB, RB, 8, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 9: return launch_one<UB, RB, 9, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 10: return launch_one<UB, RB, 10, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 11: return launch_one<UB, RB, 11, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 12:
      if constexpr (UB == 13) return launch_one<UB, RB, 12, AR, COMPOSE>(in, count, scale_exp, out, st);
      else return launch_cluster<UB, RB, 12, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 13: return launch_cluster<UB, RB, 13, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 14: return launch_cluster<UB, RB, 14, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 15:
      if constexpr (UB == 13) return launch_cluster<UB, RB, 15, AR, COMPOSE>(in, count, scale_exp, out, st);
      break;
    default: break;
  }
  return cudaErrorNotSupported;
}

template <class AR, bool COMPOSE>
cudaError_t dispatch_variant(int variant, int N, const void* in, long long count, int scale_exp, void* out,
                             cudaStream_t st) {
  switch (variant) {
    case kVariantUnit13: return dispatch_shape<13, 4, AR, COMPOSE>(N, in, count, scale_exp, out, st);
    case kVariantUnit12: return dispatch_shape<12, 4, AR, COMPOSE>(N, in, count, scale_exp, out, st);
    case kVariantUnit12x8: return dispatch_shape<12, 3, AR, COMPOSE>(N, in, count, scale_exp, out, st);
    case kVariantUnit13x8: return dispatch_shape<13, 3, AR, COMPOSE>(N, in, count, scale_exp, out, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace xk
}  // namespace pauli

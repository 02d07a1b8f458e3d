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
// Work unit: one CTA of 512 threads holds 8192 elements, 16 per thread in registers:
// 2^K consecutive masks x (the "classes", K = 13 - N) times all 2^N rows. Consecutive x
// share DRAM sectors (G[r, r^x] and G[r, r^x^1] are adjacent), and their coefficients
// n(x, z), n(x^1, z) are adjacent too, so a unit reads and writes whole sectors.
// The transform runs in 2 or 3 register phases of up to 4 butterfly stages each, with the
// data re-distributed between threads through shared memory (XOR-swizzled 16-byte slots).
//
// Arithmetic:
//  complex128: every class is converted to int64 fixed point with a per-class power-of-two
//    scale (block floating point), chosen from the class's largest exponent so that 2^N
//    terms cannot overflow; the transform is then exact (integer adds), and the only
//    roundings are the input quantisation (< 2^(N-62) max|G| per coefficient) and the final
//    correctly rounded conversion back to FP64. No FP64 instruction is used: on GB300 the
//    FP64 pipe issues ~2 ops/clk/SM while the integer pipes issue ~128.
//  complex64: TwoSum-compensated FP32: each value is an unevaluated pair (hi, lo); every
//    butterfly adds with TwoSum and carries the exact rounding error into lo.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace pauli {
namespace {

constexpr int kThreads = 512;
constexpr int kUnitBits = 13;  // 8192 elements per CTA
constexpr uint32_t kUnit = 1u << kUnitBits;

// Shared-memory slot swizzle: the low 3 bits of a 16-byte slot index are XORed with a
// linear function of its higher bits. The columns were chosen so that in every exchange
// of every layout below the 8 lanes of each quarter-warp touch 8 distinct bank groups.
__host__ __device__ constexpr uint32_t swz_col(int p) {
  return p == 3 ? 7u : p == 4 ? 5u : p == 5 ? 2u : p == 6 ? 5u : p == 7 ? 1u : p == 8 ? 5u : p == 9 ? 6u
       : p == 10 ? 6u : p == 11 ? 4u : p == 12 ? 5u : 0u;
}
__host__ __device__ constexpr uint32_t swz_term(uint32_t u) {
  uint32_t f = 0;
  for (int p = 3; p < kUnitBits; ++p)
    if ((u >> p) & 1u) f ^= swz_col(p);
  return f;
}

// Layout of a unit for L transformed row bits and K = 13 - L class bits. Element index
// u = class | (row << K). Phase p transforms the row bits [gstart, gstart + gcount); its
// registers hold those bits (padded with the lowest other row bits), its 9 thread-index
// bits hold the remaining u bits in ascending order, so lanes always vary the class bits
// first: coalesced sectors on load and store.
template <int L>
struct Layout {
  static constexpr int K = kUnitBits - L;
  static constexpr int NPH = L >= 9 ? 3 : 2;
  __host__ __device__ static constexpr int gstart(int p) { return L >= 9 ? (p == 0 ? 8 : (p == 1 ? 0 : 4)) : (p == 0 ? 4 : 0); }
  __host__ __device__ static constexpr int gcount(int p) { return L >= 9 ? (p == 0 ? L - 8 : 4) : (p == 0 ? L - 4 : 4); }
  __host__ __device__ static constexpr bool in_group(int p, int b) { return b >= gstart(p) && b < gstart(p) + gcount(p); }
  __host__ __device__ static constexpr int regpos(int p, int k) {
    if (k < gcount(p)) return K + gstart(p) + k;
    int need = k - gcount(p);
    for (int b = 0; b < L; ++b)
      if (!in_group(p, b)) {
        if (need == 0) return K + b;
        --need;
      }
    return -1;
  }
  __host__ __device__ static constexpr bool is_reg(int p, int pos) {
    for (int k = 0; k < 4; ++k)
      if (regpos(p, k) == pos) return true;
    return false;
  }
  __host__ __device__ static constexpr int thrpos(int p, int k) {
    int need = k;
    for (int pos = 0; pos < kUnitBits; ++pos)
      if (!is_reg(p, pos)) {
        if (need == 0) return pos;
        --need;
      }
    return -1;
  }
  __host__ __device__ static constexpr uint32_t reg_u(int p, int j) {
    uint32_t u = 0;
    for (int k = 0; k < 4; ++k)
      if ((j >> k) & 1) u |= 1u << regpos(p, k);
    return u;
  }
  __device__ static __forceinline__ uint32_t thread_u(int p, uint32_t t) {
    uint32_t u = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) u |= ((t >> k) & 1u) << thrpos(p, k);
    return u;
  }
};

// ---------------------------------------------------------------------- arithmetic policies
struct ArC128 {
  using Raw = longlong2;  // bit patterns of (re, im)
  struct Elem {
    long long re, im;
  };
  static constexpr bool kScaled = true;
  __device__ static __forceinline__ Raw load(const void* p, unsigned long long i) {
    return __ldg(reinterpret_cast<const longlong2*>(p) + i);
  }
  __device__ static __forceinline__ int exponent(const Raw& r) {
    return max(f64_exponent_field((uint64_t)r.x), f64_exponent_field((uint64_t)r.y));
  }
  __device__ static __forceinline__ Elem convert(const Raw& r, int s) {
    return Elem{f64_to_fixed((uint64_t)r.x, s), f64_to_fixed((uint64_t)r.y, s)};
  }
  __device__ static __forceinline__ void bfly(Elem& a, Elem& b) {
    const long long r0 = a.re + b.re, r1 = a.re - b.re, i0 = a.im + b.im, i1 = a.im - b.im;
    a.re = r0;
    a.im = i0;
    b.re = r1;
    b.im = i1;
  }
  __device__ static __forceinline__ void phase(Elem& a, uint32_t k) { mul_i_pow(a.re, a.im, k); }
  __device__ static __forceinline__ uint4 pack(const Elem& a) {
    return make_uint4((uint32_t)a.re, (uint32_t)((unsigned long long)a.re >> 32), (uint32_t)a.im,
                      (uint32_t)((unsigned long long)a.im >> 32));
  }
  __device__ static __forceinline__ Elem unpack(const uint4& q) {
    return Elem{(long long)(((unsigned long long)q.y << 32) | q.x), (long long)(((unsigned long long)q.w << 32) | q.z)};
  }
  __device__ static __forceinline__ void store(void* p, unsigned long long i, const Elem& a, int scale, bool nan) {
    double2 o;
    o.x = nan ? f64_nan() : fixed_to_f64(a.re, scale);
    o.y = nan ? f64_nan() : fixed_to_f64(a.im, scale);
    reinterpret_cast<double2*>(p)[i] = o;
  }
};

struct ArC64 {
  using Raw = float2;
  struct Elem {
    float rh, rl, ih, il;
  };
  static constexpr bool kScaled = false;
  __device__ static __forceinline__ Raw load(const void* p, unsigned long long i) {
    return __ldg(reinterpret_cast<const float2*>(p) + i);
  }
  __device__ static __forceinline__ int exponent(const Raw&) { return 0; }
  __device__ static __forceinline__ Elem convert(const Raw& r, int) { return Elem{r.x, 0.f, r.y, 0.f}; }
  __device__ static __forceinline__ void bfly(Elem& a, Elem& b) {
    float s0, e0, s1, e1, t0, f0, t1, f1;
    two_sum(a.rh, b.rh, s0, e0);
    two_sum(a.rh, -b.rh, s1, e1);
    two_sum(a.ih, b.ih, t0, f0);
    two_sum(a.ih, -b.ih, t1, f1);
    const float l0 = __fadd_rn(__fadd_rn(a.rl, b.rl), e0), l1 = __fadd_rn(__fsub_rn(a.rl, b.rl), e1);
    const float m0 = __fadd_rn(__fadd_rn(a.il, b.il), f0), m1 = __fadd_rn(__fsub_rn(a.il, b.il), f1);
    a = Elem{s0, l0, t0, m0};
    b = Elem{s1, l1, t1, m1};
  }
  __device__ static __forceinline__ void phase(Elem& a, uint32_t k) {
    mul_i_pow(a.rh, a.ih, k);
    mul_i_pow(a.rl, a.il, k);
  }
  __device__ static __forceinline__ uint4 pack(const Elem& a) {
    return make_uint4(__float_as_uint(a.rh), __float_as_uint(a.rl), __float_as_uint(a.ih), __float_as_uint(a.il));
  }
  __device__ static __forceinline__ Elem unpack(const uint4& q) {
    return Elem{__uint_as_float(q.x), __uint_as_float(q.y), __uint_as_float(q.z), __uint_as_float(q.w)};
  }
  __device__ static __forceinline__ void store(void* p, unsigned long long i, const Elem& a, int scale, bool) {
    const float f = __int_as_float((127 + scale) << 23);  // 2^scale, exact
    reinterpret_cast<float2*>(p)[i] =
        make_float2(__fmul_rn(__fadd_rn(a.rh, a.rl), f), __fmul_rn(__fadd_rn(a.ih, a.il), f));
  }
};

// Butterflies over the low G register-index bits.
template <class AR, int G>
__device__ __forceinline__ void wht_regs(typename AR::Elem (&v)[16]) {
#pragma unroll
  for (int b = 0; b < G; ++b)
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (!((j >> b) & 1)) AR::bfly(v[j], v[j | (1 << b)]);
}

template <class LY, class AR, int P>
__device__ __forceinline__ void exchange(typename AR::Elem (&v)[16], uint4* xbuf, uint32_t t, bool sync_first) {
  if (sync_first) __syncthreads();
  const uint32_t ut = LY::thread_u(P, t);
  const uint32_t ft = swz_term(ut);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const uint32_t u = ut | LY::reg_u(P, j);
    xbuf[u ^ ft ^ swz_term(LY::reg_u(P, j))] = AR::pack(v[j]);
  }
  __syncthreads();
  const uint32_t un = LY::thread_u(P + 1, t);
  const uint32_t fn = swz_term(un);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const uint32_t u = un | LY::reg_u(P + 1, j);
    v[j] = AR::unpack(xbuf[u ^ fn ^ swz_term(LY::reg_u(P + 1, j))]);
  }
}

template <int N, class AR, bool COMPOSE>
__global__ void __launch_bounds__(kThreads, 1)
    xordiag_kernel(const void* __restrict__ in, void* __restrict__ out, int scale_exp) {
  using LY = Layout<N>;
  constexpr int K = LY::K;
  constexpr uint32_t D = 1u << N;
  constexpr int LAST = LY::NPH - 1;
  extern __shared__ __align__(16) uint4 xbuf[];
  __shared__ int smax[1 << K];

  const uint32_t t = threadIdx.x;
  const unsigned long long units_per_mat = D >> K;
  const unsigned long long kmat = blockIdx.x / units_per_mat;
  const uint32_t xb = (uint32_t)(blockIdx.x % units_per_mat) << K;
  const uint32_t c = t & ((1u << K) - 1u);  // class bits are the lowest thread bits in every phase
  const uint32_t x = xb | c;
  const unsigned long long mat_elems = (unsigned long long)D * D;  // == 4^N
  const unsigned long long base = kmat * mat_elems;

  typename AR::Raw raw[16];
  int emax = 0;
  {
    const uint32_t ut = LY::thread_u(0, t);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t r = (ut | LY::reg_u(0, j)) >> K;  // row (decompose) or YZ-mask (compose)
      const unsigned long long idx =
          COMPOSE ? base + pauli_index(x, r) : base + (unsigned long long)r * D + (r ^ x);
      raw[j] = AR::load(in, idx);
      emax = max(emax, AR::exponent(raw[j]));
    }
  }
  int s = 0;
  bool nan = false;
  if (AR::kScaled) {
    if (t < (1u << K)) smax[t] = 0;
    __syncthreads();
#pragma unroll
    for (int m = 1 << K; m < 32; m <<= 1) emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, m));
    if (((t & 31u) >> K) == 0) atomicMax(&smax[c], emax);
    __syncthreads();
    const int E = smax[c];
    nan = (E == 0x7FF);
    // 2^N terms of magnitude < 2^(E-1022) * 2^s must stay below 2^62.
    s = (E == 0 || nan) ? 0 : 1084 - N - E;
  }
  typename AR::Elem v[16];
  {
    const uint32_t ut = LY::thread_u(0, t);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      v[j] = AR::convert(raw[j], s);
      if (COMPOSE) {
        const uint32_t z = (ut | LY::reg_u(0, j)) >> K;
        AR::phase(v[j], 3u * (uint32_t)__popc(x & z));  // (-i)^popc(x&z)
      }
    }
  }
  wht_regs<AR, LY::gcount(0)>(v);
  exchange<LY, AR, 0>(v, xbuf, t, false);
  wht_regs<AR, LY::gcount(1)>(v);
  if constexpr (LY::NPH == 3) {
    exchange<LY, AR, 1>(v, xbuf, t, true);
    wht_regs<AR, LY::gcount(2)>(v);
  }
  {
    const uint32_t ut = LY::thread_u(LAST, t);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t y = (ut | LY::reg_u(LAST, j)) >> K;  // YZ-mask (decompose) or row (compose)
      if (COMPOSE) {
        AR::store(out, base + (unsigned long long)y * D + (y ^ x), v[j], scale_exp - s, nan);
      } else {
        AR::phase(v[j], (uint32_t)__popc(x & y));  // i^popc(x&z)
        AR::store(out, base + pauli_index(x, y), v[j], -s - N, nan);
      }
    }
  }
}

// ------------------------------------------------------------------ N >= 13: CTA clusters --
// A class pair (x, x^1) of N > 12 qubits is 2^(N+1) elements, more than one SM holds. A
// cluster of CL = 2^(N-12) CTAs shares it: CTA q owns the rows (decompose) or YZ-masks
// (compose) whose top N-12 bits equal q, transforms their 12 low bits locally exactly as
// the N = 12 kernel does, and the remaining N-12 butterfly stages combine the CL partial
// transforms through distributed shared memory: after a cluster barrier, CTA q' reads from
// every CTA of the cluster the partial results for its slice of the low 12 output bits
// (the slice whose top log2(CL) bits equal q') and finishes the CL-point transform in
// registers. The fixed-point scale of each class is the cluster-wide maximum exponent.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t map_shared(const void* p, uint32_t rank) {
  uint32_t out;
  const uint32_t local = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(local), "r"(rank));
  return out;
}
__device__ __forceinline__ uint4 ld_dsmem16(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared::cluster.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
  return v;
}
__device__ __forceinline__ int ld_dsmem_s32(uint32_t addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

template <int N, class AR, bool COMPOSE>
__global__ void __launch_bounds__(kThreads, 1)
    xordiag_cluster_kernel(const void* __restrict__ in, void* __restrict__ out, int scale_exp) {
  using LY = Layout<12>;  // local layout: 1 class bit + 12 row bits
  constexpr int CLB = N - 12;
  constexpr uint32_t CL = 1u << CLB;
  constexpr uint32_t D = 1u << N;
  constexpr int POSB = 4 - CLB;  // log2 of output positions per thread in the combine
  static_assert(CLB >= 1 && CLB <= 3, "cluster of 2, 4 or 8 CTAs");
  extern __shared__ __align__(16) uint4 xbuf[];
  __shared__ int smax[2];

  const uint32_t t = threadIdx.x;
  const uint32_t q = cluster_rank();
  const unsigned long long unit = blockIdx.x >> CLB;  // one class pair per cluster
  const unsigned long long units_per_mat = D >> 1;
  const unsigned long long kmat = unit / units_per_mat;
  const uint32_t x = ((uint32_t)(unit % units_per_mat) << 1) | (t & 1u);
  const unsigned long long base = kmat * (unsigned long long)D * D;
  const uint32_t qoff = q << 12;

  typename AR::Raw raw[16];
  int emax = 0;
  {
    const uint32_t ut = LY::thread_u(0, t);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const uint32_t r = qoff | ((ut | LY::reg_u(0, j)) >> 1);
      const unsigned long long idx =
          COMPOSE ? base + pauli_index(x, r) : base + (unsigned long long)r * D + (r ^ x);
      raw[j] = AR::load(in, idx);
      emax = max(emax, AR::exponent(raw[j]));
    }
  }
  int s = 0;
  bool nan = false;
  if constexpr (AR::kScaled) {
    if (t < 2) smax[t] = 0;
    __syncthreads();
#pragma unroll
    for (int m = 2; m < 32; m <<= 1) emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, m));
    if ((t & 31u) < 2) atomicMax(&smax[t & 1u], emax);
    cluster_sync_all();  // every CTA's smax is final
    int E = 0;
#pragma unroll
    for (uint32_t r = 0; r < CL; ++r) E = max(E, ld_dsmem_s32(map_shared(&smax[t & 1u], r)));
    nan = (E == 0x7FF);
    s = (E == 0 || nan) ? 0 : 1084 - N - E;
  }
  typename AR::Elem v[16];
  {
    const uint32_t ut = LY::thread_u(0, t);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      v[j] = AR::convert(raw[j], s);
      if (COMPOSE) {
        const uint32_t z = qoff | ((ut | LY::reg_u(0, j)) >> 1);
        AR::phase(v[j], 3u * (uint32_t)__popc(x & z));
      }
    }
  }
  wht_regs<AR, 4>(v);
  exchange<LY, AR, 0>(v, xbuf, t, false);
  wht_regs<AR, 4>(v);
  exchange<LY, AR, 1>(v, xbuf, t, true);
  wht_regs<AR, 4>(v);
  // publish the local transform
  __syncthreads();
  {
    const uint32_t ut = LY::thread_u(2, t);
    const uint32_t ft = swz_term(ut);
#pragma unroll
    for (int j = 0; j < 16; ++j) xbuf[ut ^ LY::reg_u(2, j) ^ ft ^ swz_term(LY::reg_u(2, j))] = AR::pack(v[j]);
  }
  cluster_sync_all();
  // combine: lane bits (class, y0..y3), warp bits y4..y7, POSB position bits y8.., rank bits on top
  const uint32_t lane_part = ((t >> 1) & 15u) | (((t >> 5) & 15u) << 4);
#pragma unroll
  for (int p = 0; p < (1 << POSB); ++p) {
    const uint32_t yl = lane_part | ((uint32_t)p << 8) | (q << (12 - CLB));  // low 12 output bits
    const uint32_t u = (t & 1u) | (yl << 1);
    const uint32_t slot = u ^ swz_term(u);
    typename AR::Elem w[CL];
#pragma unroll
    for (uint32_t r = 0; r < CL; ++r) w[r] = AR::unpack(ld_dsmem16(map_shared(&xbuf[slot], r)));
#pragma unroll
    for (int b = 0; b < CLB; ++b)
#pragma unroll
      for (uint32_t r = 0; r < CL; ++r)
        if (!((r >> b) & 1u)) AR::bfly(w[r], w[r | (1u << b)]);
#pragma unroll
    for (uint32_t r = 0; r < CL; ++r) {
      const uint32_t y = yl | (r << 12);  // YZ-mask (decompose) or row (compose)
      if (COMPOSE) {
        AR::store(out, base + (unsigned long long)y * D + (y ^ x), w[r], scale_exp - s, nan);
      } else {
        AR::phase(w[r], (uint32_t)__popc(x & y));
        AR::store(out, base + pauli_index(x, y), w[r], -s - N, nan);
      }
    }
  }
  cluster_sync_all();  // peers may still be reading this CTA's shared memory
}

template <int N, class AR, bool COMPOSE>
cudaError_t launch_cluster(const void* in, long long count, int scale_exp, void* out, cudaStream_t st) {
  constexpr size_t smem = (size_t)kUnit * 16;
  constexpr unsigned CL = 1u << (N - 12);
  auto kern = xordiag_cluster_kernel<N, AR, COMPOSE>;
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const unsigned long long ctas = (unsigned long long)count * ((1ull << N) >> 1) * CL;
  if (ctas > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, in, out, scale_exp);
}

template <int N, class AR, bool COMPOSE>
cudaError_t launch_one(const void* in, long long count, int scale_exp, void* out, cudaStream_t st) {
  constexpr size_t smem = (size_t)kUnit * 16;
  auto kern = xordiag_kernel<N, AR, COMPOSE>;
  static bool attr_done = false;  // one device per process in this library
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  const unsigned long long units = (unsigned long long)count * ((1ull << (2 * N)) >> kUnitBits);
  if (units > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
  kern<<<(unsigned)units, kThreads, smem, st>>>(in, out, scale_exp);
  return cudaGetLastError();
}

template <class AR, bool COMPOSE>
cudaError_t dispatch_n(int N, const void* in, long long count, int scale_exp, void* out, cudaStream_t st) {
  switch (N) {
    case 7: return launch_one<7, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 8: return launch_one<8, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 9: return launch_one<9, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 10: return launch_one<10, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 11: return launch_one<11, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 12: return launch_one<12, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 13: return launch_cluster<13, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 14: return launch_cluster<14, AR, COMPOSE>(in, count, scale_exp, out, st);
    case 15: return launch_cluster<15, AR, COMPOSE>(in, count, scale_exp, out, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

bool xordiag_supported(int N) { return N >= 7 && N <= 15; }

cudaError_t launch_xordiag(const void* in, int N, long long count, bool c64, bool compose, int scale_exp, void* out,
                           cudaStream_t s) {
  if (c64)
    return compose ? dispatch_n<ArC64, true>(N, in, count, scale_exp, out, s)
                   : dispatch_n<ArC64, false>(N, in, count, scale_exp, out, s);
  return compose ? dispatch_n<ArC128, true>(N, in, count, scale_exp, out, s)
                 : dispatch_n<ArC128, false>(N, in, count, scale_exp, out, s);
}

}  // namespace pauli

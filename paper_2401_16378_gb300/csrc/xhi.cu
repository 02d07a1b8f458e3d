// xhi.cu -- decomposition of one x-class shard: the coefficients whose XY-mask x has the top
// k bits x_hi, from the 2^k blocks of G that hold them.
//
// Write r = (r_hi, r_lo), x = (x_hi, x_lo), z = (z_hi, z_lo) with the top k bits first and
// m = N - k. In the XOR-diagonal form of Eq. (13),
//   c(x, z) = 2^-N i^popc(x & z) sum_r (-1)^popc(r & z) G[r, r ^ x],
// the element G[r, r ^ x] lies in block (r_hi, r_hi ^ x_hi) of G (blocks of 2^m x 2^m), at
// (r_lo, r_lo ^ x_lo) inside it. Splitting the sum over r and the phase over the two halves,
//   c(x, z) = 2^-k i^popc(x_hi & z_hi) sum_{r_hi} (-1)^popc(r_hi & z_hi) c_{B(r_hi)}(x_lo, z_lo),
// where B(r_hi) is the m-qubit block (r_hi, r_hi ^ x_hi) and c_B its own coefficients. The Pauli
// index is interleaved per qubit (Eq. (2)), so c_B's index n_lo = n(x_lo, z_lo) is the low 2m
// bits of n(x, z). The shard is therefore computed as
//  1. the m-qubit decomposition of the 2^k blocks, stacked by r_hi (one batched pauli_decompose
//     into out: out[r_hi 4^m + n_lo] = c_{B(r_hi)}(n_lo)), then
//  2. in place, a k-bit Walsh-Hadamard transform over r_hi at every n_lo, the phase
//     i^popc(x_hi & z_hi) and the exact scale 2^-k: out[z_hi 4^m + n_lo] = c(x, z).
// For N = 12..14 with m >= 6 the two-stage kernel instead runs the whole transform of the shard's
// classes in one launch, reading the layout's tiles and writing the compact index directly
// (twostage_impl.cuh, ShardArgs): the same arithmetic, bit for bit, as the full decomposition.
// Step 2 runs in passes of up to 4 bits of r_hi (registers hold 2^4 values), the phase and
// scale in the last pass. Its sums are FP64 for both dtypes (complex64 values are widened and
// rounded once per pass).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"

namespace pauli {
namespace {

template <bool C64>
struct XhiElem {
  using T = double2;
  __device__ static __forceinline__ double2 load(const void* p, unsigned long long i) {
    return __ldcs(static_cast<const double2*>(p) + i);
  }
  __device__ static __forceinline__ void store(void* p, unsigned long long i, double2 v) {
    __stcs(static_cast<double2*>(p) + i, v);
  }
};
template <>
struct XhiElem<true> {
  __device__ static __forceinline__ double2 load(const void* p, unsigned long long i) {
    const float2 f = __ldcs(static_cast<const float2*>(p) + i);
    return make_double2((double)f.x, (double)f.y);
  }
  __device__ static __forceinline__ void store(void* p, unsigned long long i, double2 v) {
    __stcs(static_cast<float2*>(p) + i, make_float2(__double2float_rn(v.x), __double2float_rn(v.y)));
  }
};

// One pass over bits [b0, b0 + B) of r_hi. Thread work item w < 4^m 2^(k - B): n_lo = w mod 4^m,
// the other r_hi bits from w >> 2m. LAST: apply i^popc(x_hi & z_hi) and 2^-k.
template <int B, bool C64, bool LAST>
__global__ void __launch_bounds__(256) xhi_combine(void* __restrict__ out, int m2, int k, int b0, uint32_t x_hi,
                                                   double scale, unsigned long long items) {
  using EL = XhiElem<C64>;
  const unsigned long long lo_mask = (1ull << m2) - 1ull;
  for (unsigned long long w = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; w < items;
       w += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long n_lo = w & lo_mask;
    const uint32_t rest = (uint32_t)(w >> m2);  // r_hi bits outside the group, low ones first
    const uint32_t below = rest & ((1u << b0) - 1u);
    const uint32_t hi = (rest >> b0) << (b0 + B);
    double2 v[1 << B];
#pragma unroll
    for (int j = 0; j < (1 << B); ++j) {
      const uint32_t rh = hi | ((uint32_t)j << b0) | below;
      v[j] = EL::load(out, ((unsigned long long)rh << m2) | n_lo);
    }
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int j = 0; j < (1 << B); ++j)
        if (!((j >> b) & 1)) {
          const double2 a = v[j], c = v[j | (1 << b)];
          v[j] = make_double2(a.x + c.x, a.y + c.y);
          v[j | (1 << b)] = make_double2(a.x - c.x, a.y - c.y);
        }
#pragma unroll
    for (int j = 0; j < (1 << B); ++j) {
      const uint32_t zh = hi | ((uint32_t)j << b0) | below;  // after the transform: the z_hi index
      double2 o = v[j];
      if (LAST) {
        double re = o.x * scale, im = o.y * scale;
        mul_i_pow(re, im, (uint32_t)__popc(x_hi & zh));
        o = make_double2(re, im);
      }
      EL::store(out, ((unsigned long long)zh << m2) | n_lo, o);
    }
  }
}

template <int B, bool C64>
cudaError_t launch_pass(void* out, int m, int k, int b0, bool last, uint32_t x_hi, cudaStream_t s) {
  const unsigned long long items = (1ull << (2 * m)) << (k - B);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const unsigned long long want = (items + 255) / 256;
  const unsigned long long cap = (unsigned long long)sms * 8ull;  // 8 CTAs of 256 threads per SM
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  const double scale = ldexp(1.0, -k);
  if (last)
    xhi_combine<B, C64, true><<<grid, 256, 0, s>>>(out, 2 * m, k, b0, x_hi, scale, items);
  else
    xhi_combine<B, C64, false><<<grid, 256, 0, s>>>(out, 2 * m, k, b0, x_hi, scale, items);
  return cudaGetLastError();
}

template <bool C64>
cudaError_t launch_pass_b(int B, void* out, int m, int k, int b0, bool last, uint32_t x_hi, cudaStream_t s) {
  switch (B) {
    case 1: return launch_pass<1, C64>(out, m, k, b0, last, x_hi, s);
    case 2: return launch_pass<2, C64>(out, m, k, b0, last, x_hi, s);
    case 3: return launch_pass<3, C64>(out, m, k, b0, last, x_hi, s);
    default: return launch_pass<4, C64>(out, m, k, b0, last, x_hi, s);
  }
}

}  // namespace

cudaError_t twostage_launch_xhi_c128(const void* L, int N, int k, uint32_t x_hi, void* out, cudaStream_t st);
cudaError_t twostage_launch_xhi_c64(const void* L, int N, int k, uint32_t x_hi, void* out, cudaStream_t st);

cudaError_t twostage_launch_xhi(const void* L, int N, int k, uint32_t x_hi, bool c64, void* out, cudaStream_t s) {
  if (N < 12 || N > 14 || N - k < 6 || (reinterpret_cast<uintptr_t>(L) & 15u)) return cudaErrorNotSupported;
  return c64 ? twostage_launch_xhi_c64(L, N, k, x_hi, out, s) : twostage_launch_xhi_c128(L, N, k, x_hi, out, s);
}

cudaError_t launch_xhi_combine(void* out, int N, int k, uint32_t x_hi, bool c64, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  const int m = N - k;
  // passes of 4 bits from the bottom; the last (possibly shorter) one applies phase and scale
  for (int b0 = 0; b0 < k; b0 += 4) {
    const int B = k - b0 < 4 ? k - b0 : 4;
    const bool last = b0 + B == k;
    cudaError_t e = c64 ? launch_pass_b<true>(B, out, m, k, b0, last, x_hi, s)
                        : launch_pass_b<false>(B, out, m, k, b0, last, x_hi, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace {

// L[r][j] = G[r][((r_hi ^ x_hi) << m) | j], moved in words of W bytes: word w of row r of L
// (rows of M elements = rw words) comes from the same word of the row's block in G.
template <class W>
__global__ void __launch_bounds__(256) xhi_layout_kernel(const char* __restrict__ G, char* __restrict__ L, int N,
                                                         int m, uint32_t x_hi, size_t elem, int rw_log,
                                                         unsigned long long words) {
  const unsigned long long row_bytes = (unsigned long long)elem << N;
  const unsigned long long rw_mask = (1ull << rw_log) - 1ull;  // rows of L hold 2^rw_log words
  for (unsigned long long w = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; w < words;
       w += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long r = w >> rw_log, c = w & rw_mask;
    const unsigned long long cb = ((r >> m) ^ x_hi) << m;  // first column of the row's block
    const W v = __ldcs(reinterpret_cast<const W*>(G + r * row_bytes + cb * elem) + c);
    __stcs(reinterpret_cast<W*>(L) + w, v);
  }
}

}  // namespace

cudaError_t xhi_layout(const void* G, int N, int k, uint32_t x_hi, size_t elem, void* L, cudaStream_t s) {
  const int m = N - k;
  const unsigned long long bytes = (unsigned long long)elem << (2 * N - k);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // 16-byte words when both buffers allow them (a row of L is at least 16 bytes: m >= 1)
  const bool wide = !((reinterpret_cast<uintptr_t>(G) | reinterpret_cast<uintptr_t>(L)) & 15u);
  const unsigned long long words = bytes / (wide ? 16u : elem);
  const unsigned long long want = (words + 255) / 256, cap = (unsigned long long)sms * 8ull;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  const char* g = static_cast<const char*>(G);
  char* l = static_cast<char*>(L);
  const int elog = elem == 16 ? 4 : 3;
  // words per row of L: 2^m elements of 2^elog bytes in words of 16 bytes or of one element
  const int rw_log = m + elog - (wide ? 4 : elog);
  if (wide)
    xhi_layout_kernel<uint4><<<grid, 256, 0, s>>>(g, l, N, m, x_hi, elem, rw_log, words);
  else if (elem == 16)
    xhi_layout_kernel<double2><<<grid, 256, 0, s>>>(g, l, N, m, x_hi, elem, rw_log, words);
  else
    xhi_layout_kernel<float2><<<grid, 256, 0, s>>>(g, l, N, m, x_hi, elem, rw_log, words);
  return cudaGetLastError();
}

}  // namespace pauli

// plain.cu -- the paper's per-coefficient sum (Eq. (13)) on the GPU.
//
// Each coefficient c(x, z) = 2^-N i^popc(x&z) sum_r (-1)^popc(r&z) G[r, r^x] is an O(2^N)
// sum (Sec. 3: O(2^N) per coefficient, O(8^N) for all 4^N). A warp owns a tile of
// CW <= 8 XY-masks x (consecutive, so that the lanes of one row read CW adjacent
// elements: coalesced 16-byte loads) times KZ <= 8 YZ-masks z, and splits the rows r into
// RS = 32 / CW interleaved subsets, one per lane group. Each lane visits its rows in
// Gray-code order and keeps the KZ signs (-1)^popc(r&z) as a bit mask that flips by one
// precomputed pattern per step -- the recurrence of Eq. (14), where a Gray step changes one
// bit t of r and the sign of every z with bit t set. The RS partial sums are combined with
// warp shuffles in FP64.
//
// complex128: FP64 accumulation. complex64: TwoSum-compensated FP32 accumulation per lane
// (s, e) with e collecting the exact rounding error of every addition; the partial sums
// are widened to FP64 for the cross-lane reduction and rounded to FP32 once at the end.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace pauli {

namespace {

constexpr int kWarpsPerBlock = 8;

// Bit pattern over k in [0, 8) of "bit b of k is set".
__device__ __forceinline__ uint32_t k_pattern(int b) {
  return b == 0 ? 0xAAu : (b == 1 ? 0xCCu : 0xF0u);
}

struct AccC128 {
  double re[8], im[8];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < 8; ++k) re[k] = im[k] = 0.0;
  }
  __device__ __forceinline__ void add(int k, double vr, double vi, uint32_t neg) {
    const long long flip = (long long)neg << 63;
    re[k] += __longlong_as_double(__double_as_longlong(vr) ^ flip);
    im[k] += __longlong_as_double(__double_as_longlong(vi) ^ flip);
  }
  __device__ __forceinline__ double total_re(int k) const { return re[k]; }
  __device__ __forceinline__ double total_im(int k) const { return im[k]; }
};

struct AccC64 {
  float sr[8], er[8], si[8], ei[8];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int k = 0; k < 8; ++k) sr[k] = er[k] = si[k] = ei[k] = 0.f;
  }
  __device__ __forceinline__ void add(int k, float vr, float vi, uint32_t neg) {
    const int flip = (int)(neg << 31);
    vr = __int_as_float(__float_as_int(vr) ^ flip);
    vi = __int_as_float(__float_as_int(vi) ^ flip);
    float s, e;
    two_sum(sr[k], vr, s, e);
    sr[k] = s;
    er[k] = __fadd_rn(er[k], e);
    two_sum(si[k], vi, s, e);
    si[k] = s;
    ei[k] = __fadd_rn(ei[k], e);
  }
  __device__ __forceinline__ double total_re(int k) const { return (double)sr[k] + (double)er[k]; }
  __device__ __forceinline__ double total_im(int k) const { return (double)si[k] + (double)ei[k]; }
};

// RE: store only Re c_n, into an array of reals (Hermitian decomposition). UPPER (with RE): G is
// Hermitian and read from its upper triangle; an element below the diagonal, G[r, r ^ x] with
// bit h of r set (h the top set bit of x), is read as conj(G[r ^ x, r]).
// REALIN (complex128 arithmetic, with RE): G is a real float64 matrix; the output is the real
// a_n with c_n = i^(k mod 2) a_n, k = popc(x & z) the number of Y factors.
// WS > 1 (small grids): the WS warps of a block share one tile and take consecutive runs of
// its Gray steps; their partial sums meet in shared memory, added in warp order.
template <bool C64, bool RE, bool UPPER = false, bool REALIN = false>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) plain_decompose_kernel(const void* __restrict__ Gv, int N,
                                                                             long long count, void* __restrict__ outv,
                                                                             int WS) {
  using Acc = typename std::conditional<C64, AccC64, AccC128>::type;
  const uint32_t D = 1u << N;
  const int lcw = N < 3 ? N : 3;  // log2 CW
  const int lkz = N < 3 ? N : 3;  // log2 KZ
  const uint32_t CW = 1u << lcw, KZ = 1u << lkz;
  const int lrs = (5 - lcw) < N ? (5 - lcw) : N;  // log2 RS, at most N
  const uint32_t RS = 1u << lrs;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t c = lane & (CW - 1u);
  const uint32_t rsub = lane >> lcw;
  const bool active = rsub < RS;

  const unsigned long long tiles_x = D >> lcw, tiles_z = D >> lkz;
  const unsigned long long tiles_per_mat = tiles_x * tiles_z;
  const uint32_t wchunk = WS > 1 ? threadIdx.x >> 5 : 0u;  // this warp's run of Gray steps
  const unsigned long long w =
      WS > 1 ? (unsigned long long)blockIdx.x : (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= tiles_per_mat * (unsigned long long)count) return;  // whole warp (whole block for WS > 1) leaves together
  const unsigned long long kmat = w / tiles_per_mat;
  const unsigned long long tile = w % tiles_per_mat;
  const uint32_t x = (uint32_t)(tile / tiles_z) * CW + c;
  const uint32_t zb = (uint32_t)(tile % tiles_z) * KZ;

  const uint32_t hx = x ? 31u - (uint32_t)__clz(x) : 32u;  // top set bit of x (UPPER)
  Acc acc;
  acc.zero();
  if (active) {
    const uint32_t steps_all = D >> lrs;
    const uint32_t steps = steps_all / (uint32_t)WS, gbeg = wchunk * steps;  // WS divides steps_all
    // initial signs at the first Gray step of the run (row r = rsub | gray(gbeg) << lrs)
    const uint32_t r0 = rsub | ((gbeg ^ (gbeg >> 1)) << lrs);
    uint32_t signs = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if ((uint32_t)k < KZ) signs |= (uint32_t)(__popc(r0 & (zb + k)) & 1) << k;
    const uint32_t kmask = (1u << KZ) - 1u;
    using Val = typename std::conditional<C64, float2, double2>::type;
    const unsigned long long mbase = kmat * (unsigned long long)D * D;
    // element of row r of the XOR-diagonal of x (mirrored / real input as the flags say)
    auto load = [&](uint32_t r) -> Val {
      if constexpr (REALIN) {
        return Val{__ldg(&reinterpret_cast<const double*>(Gv)[mbase + (unsigned long long)r * D + (r ^ x)]), 0.0};
      } else {
        const Val* G = reinterpret_cast<const Val*>(Gv) + mbase;
        Val e;
        if (UPPER && hx < 32u && ((r >> hx) & 1u)) {
          e = __ldg(&G[(unsigned long long)(r ^ x) * D + r]);
          e.y = -e.y;
        } else {
          e = __ldg(&G[(unsigned long long)r * D + (r ^ x)]);
          if (UPPER && x == 0u) e.y = 0;  // the diagonal: its imaginary parts are not used
        }
        return e;
      }
    };
    // The loads of kBatch consecutive Gray steps are independent: issue them together, then
    // accumulate in step order (the sign recurrence and the sums keep their sequence).
    constexpr uint32_t kBatch = 4;
    for (uint32_t g0 = gbeg; g0 < gbeg + steps; g0 += kBatch) {
      Val e[kBatch];
#pragma unroll
      for (uint32_t u = 0; u < kBatch; ++u) {
        const uint32_t g = g0 + u;
        if (g < gbeg + steps) e[u] = load(rsub | ((g ^ (g >> 1)) << lrs));
      }
#pragma unroll
      for (uint32_t u = 0; u < kBatch; ++u) {
        const uint32_t g = g0 + u;
        if (g >= gbeg + steps) break;
        if (g != gbeg) {
          const int zbit = __ffs(g) - 1 + lrs;  // row bit changed by this Gray step
          const uint32_t flip = zbit < lkz ? k_pattern(zbit) : (((zb >> zbit) & 1u) ? 0xFFu : 0u);
          signs ^= flip & kmask;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if ((uint32_t)k < KZ) acc.add(k, e[u].x, e[u].y, (signs >> k) & 1u);
      }
    }
  }
  // FP64 reduction over the RS row subsets (lane bits lcw .. lcw+lrs-1)
  double tr[8], ti[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    tr[k] = acc.total_re(k);
    ti[k] = acc.total_im(k);
  }
  for (uint32_t m = CW; m < (CW << lrs); m <<= 1) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      tr[k] += __shfl_xor_sync(0xFFFFFFFFu, tr[k], m);
      ti[k] += __shfl_xor_sync(0xFFFFFFFFu, ti[k], m);
    }
  }
  if (WS > 1) {  // the block's warps meet: partials of the first row subset's lanes, [warp][c][k]
    __shared__ double part[4][8][8][2];
    if (rsub == 0) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        part[wchunk][c][k][0] = tr[k];
        part[wchunk][c][k][1] = ti[k];
      }
    }
    __syncthreads();
    if (wchunk != 0) return;
    if (rsub == 0) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        tr[k] = part[0][c][k][0];
        ti[k] = part[0][c][k][1];
        for (int q = 1; q < WS; ++q) {
          tr[k] += part[q][c][k][0];
          ti[k] += part[q][c][k][1];
        }
      }
    }
  }
  if (rsub != 0) return;
  const double scale = 1.0 / (double)D;  // exact power of two
  const unsigned long long nco = (unsigned long long)D * D;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if ((uint32_t)k >= KZ) break;
    const uint32_t z = zb + k;
    double re = tr[k] * scale, im = ti[k] * scale;
    mul_i_pow(re, im, (uint32_t)__popc(x & z));
    const unsigned long long n = kmat * nco + pauli_index(x, z);
    if (REALIN) {
      reinterpret_cast<double*>(outv)[n] = (__popc(x & z) & 1) ? im : re;
    } else if (RE) {
      if (C64)
        reinterpret_cast<float*>(outv)[n] = (float)re;
      else
        reinterpret_cast<double*>(outv)[n] = re;
    } else if (C64) {
      reinterpret_cast<float2*>(outv)[n] = make_float2((float)re, (float)im);
    } else {
      reinterpret_cast<double2*>(outv)[n] = make_double2(re, im);
    }
  }
}

// One warp per listed coefficient; lanes split the rows and reduce with shuffles.
template <bool C64>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) coeffs_at_kernel(const void* __restrict__ Gv, int N,
                                                                       const uint64_t* __restrict__ idx, long long k,
                                                                       void* __restrict__ outv) {
  const unsigned long long q = (unsigned long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  if (q >= (unsigned long long)k) return;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t D = 1u << N;
  const uint64_t n = idx[q];
  const bool valid = n < ((uint64_t)1 << (2 * N));
  uint32_t x = 0, z = 0;
  pauli_xz((uint32_t)n, x, z);
  const int lrs = N < 5 ? N : 5;
  const uint32_t RS = 1u << lrs;
  double tr = 0.0, ti = 0.0;
  if (valid && lane < RS) {
    const uint32_t steps = D >> lrs;
    if (C64) {
      const float2* G = reinterpret_cast<const float2*>(Gv);
      AccC64 a;
      a.zero();
      for (uint32_t g = 0; g < steps; ++g) {
        const uint32_t r = lane | (g << lrs);
        const float2 e = __ldg(&G[(unsigned long long)r * D + (r ^ x)]);
        a.add(0, e.x, e.y, (uint32_t)__popc(r & z) & 1u);
      }
      tr = a.total_re(0);
      ti = a.total_im(0);
    } else {
      const double2* G = reinterpret_cast<const double2*>(Gv);
      AccC128 a;
      a.re[0] = a.im[0] = 0.0;
      for (uint32_t g = 0; g < steps; ++g) {
        const uint32_t r = lane | (g << lrs);
        const double2 e = __ldg(&G[(unsigned long long)r * D + (r ^ x)]);
        a.add(0, e.x, e.y, (uint32_t)__popc(r & z) & 1u);
      }
      tr = a.re[0];
      ti = a.im[0];
    }
  }
#pragma unroll
  for (int m = 1; m < 32; m <<= 1) {
    tr += __shfl_xor_sync(0xFFFFFFFFu, tr, m);
    ti += __shfl_xor_sync(0xFFFFFFFFu, ti, m);
  }
  if (lane != 0) return;
  double re = tr / (double)D, im = ti / (double)D;
  mul_i_pow(re, im, (uint32_t)__popc(x & z));
  if (!valid) re = im = f64_nan();
  if (C64)
    reinterpret_cast<float2*>(outv)[q] = make_float2((float)re, (float)im);
  else
    reinterpret_cast<double2*>(outv)[q] = make_double2(re, im);
}


// Eq. (1) elementwise: G[r, q] = 2^scale_exp sum_z (-1)^popc(r&z) (-i)^popc(x&z) c(x, z) with
// x = r ^ q -- only the 2^N tensors whose XY-mask equals r ^ q have a nonzero entry at (r, q)
// (Eq. (8), (11)). One thread per matrix element, O(2^N) each. With weights wv (nullable),
// each c_n is first multiplied by g w_n (g = *gv, or 1 when gv is null).
template <bool C64>
__global__ void __launch_bounds__(256) plain_compose_kernel(const void* __restrict__ cv, int N, long long count,
                                                            int scale_exp, void* __restrict__ Gv,
                                                            const void* __restrict__ wv, const void* __restrict__ gv) {
  const unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t D = 1u << N;
  const unsigned long long per = (unsigned long long)D * D;
  if (e >= per * (unsigned long long)count) return;
  const unsigned long long kmat = e / per;
  const uint32_t r = (uint32_t)((e % per) >> N), q = (uint32_t)(e % per) & (D - 1u);
  const uint32_t x = r ^ q;
  double tr = 0.0, ti = 0.0;
  if (C64) {
    const float2* c = reinterpret_cast<const float2*>(cv) + kmat * per;
    const float* w = static_cast<const float*>(wv);
    const float g = gv ? *static_cast<const float*>(gv) : 1.0f;
    AccC64 a;
    a.zero();
    for (uint32_t z = 0; z < D; ++z) {
      const uint32_t n = pauli_index(x, z);
      const float2 v = __ldg(&c[n]);
      float vr = v.x, vi = v.y;
      if (w) {
        const float f = g == 1.0f ? w[n] : g * w[n];
        vr *= f;
        vi *= f;
      }
      mul_i_pow(vr, vi, 3u * (uint32_t)__popc(x & z));
      a.add(0, vr, vi, (uint32_t)__popc(r & z) & 1u);
    }
    tr = a.total_re(0);
    ti = a.total_im(0);
  } else {
    const double2* c = reinterpret_cast<const double2*>(cv) + kmat * per;
    const double* w = static_cast<const double*>(wv);
    const double g = gv ? *static_cast<const double*>(gv) : 1.0;
    for (uint32_t z = 0; z < D; ++z) {
      const uint32_t n = pauli_index(x, z);
      const double2 v = __ldg(&c[n]);
      double vr = v.x, vi = v.y;
      if (w) {
        const double f = g == 1.0 ? w[n] : g * w[n];
        vr *= f;
        vi *= f;
      }
      mul_i_pow(vr, vi, 3u * (uint32_t)__popc(x & z));
      const long long flip = (long long)(__popc(r & z) & 1) << 63;
      tr += __longlong_as_double(__double_as_longlong(vr) ^ flip);
      ti += __longlong_as_double(__double_as_longlong(vi) ^ flip);
    }
  }
  const double f = ldexp(1.0, scale_exp);
  if (C64)
    reinterpret_cast<float2*>(Gv)[e] = make_float2((float)(tr * f), (float)(ti * f));
  else
    reinterpret_cast<double2*>(Gv)[e] = make_double2(tr * f, ti * f);
}

}  // namespace

// Warps per block of the plain kernels: one for small grids, so that the blocks (and their FP64
// work) spread over the SMs -- at N = 6 the 64 warps of a matrix would otherwise share 8 SMs'
// FP64 pipes -- and kWarpsPerBlock otherwise.
static int plain_warps_per_block(unsigned long long tiles) { return tiles < 4096ull ? 1 : kWarpsPerBlock; }
// Warps sharing one tile: up to 4 for small grids (one per SM sub-partition and its FP64 unit),
// dividing the Gray steps of each lane (2^N / row subsets).
static int plain_warps_per_tile(int N, unsigned long long tiles) {
  const int lcw = N < 3 ? N : 3;
  const int lrs = (5 - lcw) < N ? (5 - lcw) : N;
  const unsigned long long steps = (1ull << N) >> lrs;
  if (tiles >= 4096ull) return 1;
  return steps >= 4 ? 4 : (int)steps;
}

cudaError_t launch_plain_decompose(const void* G, int N, long long count, bool c64, void* out, cudaStream_t s,
                                   bool re, bool upper) {
  const int lcw = N < 3 ? N : 3, lkz = lcw;
  const unsigned long long tiles = ((1ull << N) >> lcw) * ((1ull << N) >> lkz) * (unsigned long long)count;
  const int ws = plain_warps_per_tile(N, tiles);
  const int wpb = ws > 1 ? ws : plain_warps_per_block(tiles);
  const unsigned long long blocks = ws > 1 ? tiles : (tiles + wpb - 1) / wpb;
  if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
  auto kern = c64 ? (re ? (upper ? plain_decompose_kernel<true, true, true> : plain_decompose_kernel<true, true>)
                        : plain_decompose_kernel<true, false>)
                  : (re ? (upper ? plain_decompose_kernel<false, true, true> : plain_decompose_kernel<false, true>)
                        : plain_decompose_kernel<false, false>);
  kern<<<(unsigned)blocks, wpb * 32, 0, s>>>(G, N, count, out, ws);
  return cudaGetLastError();
}

cudaError_t launch_plain_decompose_real(const void* G, int N, long long count, void* out, cudaStream_t s) {
  const int lcw = N < 3 ? N : 3, lkz = lcw;
  const unsigned long long tiles = ((1ull << N) >> lcw) * ((1ull << N) >> lkz) * (unsigned long long)count;
  const int ws = plain_warps_per_tile(N, tiles);
  const int wpb = ws > 1 ? ws : plain_warps_per_block(tiles);
  const unsigned long long blocks = ws > 1 ? tiles : (tiles + wpb - 1) / wpb;
  if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
  plain_decompose_kernel<false, true, false, true><<<(unsigned)blocks, wpb * 32, 0, s>>>(G, N, count, out, ws);
  return cudaGetLastError();
}

cudaError_t launch_plain_compose(const void* c, int N, long long count, bool c64, int scale_exp, void* G,
                                cudaStream_t s, const void* w, const void* g) {
  const unsigned long long total = (1ull << (2 * N)) * (unsigned long long)count;
  const unsigned long long blocks = (total + 255) / 256;
  if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
  if (c64)
    plain_compose_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(c, N, count, scale_exp, G, w, g);
  else
    plain_compose_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(c, N, count, scale_exp, G, w, g);
  return cudaGetLastError();
}

cudaError_t launch_coeffs_at(const void* G, int N, bool c64, const uint64_t* idx, long long k, void* out,
                             cudaStream_t s) {
  const unsigned long long blocks = ((unsigned long long)k + kWarpsPerBlock - 1) / kWarpsPerBlock;
  if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidConfiguration;
  if (c64)
    coeffs_at_kernel<true><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(G, N, idx, k, out);
  else
    coeffs_at_kernel<false><<<(unsigned)blocks, kWarpsPerBlock * 32, 0, s>>>(G, N, idx, k, out);
  return cudaGetLastError();
}

}  // namespace pauli

// common.cuh -- device helpers shared by the libpauli kernels (sm_103a).
//
// Notation follows arXiv 2401.16378 (Sec. 2): N qubits, D = 2^N, Pauli index n with base-4
// digits p_t = (n >> 2t) & 3 naming I, X, Y, Z. For a tensor n define the bit masks
//   x = XY-mask (bit t set when p_t is X or Y: the mask m^(n) of Eq. (11)),
//   z = YZ-mask (bit t set when p_t is Y or Z).
// Per digit (b1 b0) = (p_t >> 1, p_t & 1): x_t = b0 ^ b1 and z_t = b1, so the even bits of n
// are x ^ z and the odd bits are z. The lambda of Eq. (12) is then
//   lambda_i = (-i)^popc(x & z) * (-1)^popc(i & z),
// because the nonzero entries of Z and Y in row a are (-1)^a and -i (-1)^a (Eq. (3), (8)).
// Substituting r = i ^ x into Eq. (13) gives
//   c(x, z) = 2^-N * i^popc(x & z) * sum_r (-1)^popc(r & z) * G[r, r ^ x],
// a Walsh-Hadamard transform over r of e_x[r] = G[r, r ^ x] (row r, column r ^ x).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pauli {

// ---------------------------------------------------------------- index codec (Eq. (2)) --
// Spread the low 16 bits of v to the even bit positions of a 32-bit word.
__device__ __forceinline__ uint32_t spread16(uint32_t v) {
  v &= 0xFFFFu;
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}
// Inverse of spread16 on the even bits of v.
__device__ __forceinline__ uint32_t compact16(uint32_t v) {
  v &= 0x55555555u;
  v = (v | (v >> 1)) & 0x33333333u;
  v = (v | (v >> 2)) & 0x0F0F0F0Fu;
  v = (v | (v >> 4)) & 0x00FF00FFu;
  v = (v | (v >> 8)) & 0x0000FFFFu;
  return v;
}
// n(x, z): even bits x ^ z, odd bits z (N <= 16, so n fits in 32 bits).
__device__ __forceinline__ uint32_t pauli_index(uint32_t x, uint32_t z) {
  return spread16(x ^ z) | (spread16(z) << 1);
}
__device__ __forceinline__ void pauli_xz(uint32_t n, uint32_t& x, uint32_t& z) {
  const uint32_t e = compact16(n), o = compact16(n >> 1);
  z = o;
  x = e ^ o;
}

// --------------------------------------------------- phases i^k on (re, im) pairs (exact) --
// Multiply (re, im) by i^k, k taken mod 4: 1 -> (-im, re), 2 -> (-re, -im), 3 -> (im, -re).
template <class T>
__device__ __forceinline__ void mul_i_pow(T& re, T& im, uint32_t k) {
  const T r = re, m = im;
  switch (k & 3u) {
    case 0: break;
    case 1: re = -m; im = r; break;
    case 2: re = -r; im = -m; break;
    default: re = m; im = -r; break;
  }
}

// ------------------------------------ FP64 <-> int64 fixed point, integer instructions only --
// The GB300 FP64 pipe issues about 2 operations per clock per SM, so the XOR-diagonal path
// keeps FP64 values as bit patterns and converts them with integer arithmetic.
__device__ __forceinline__ int f64_exponent_field(uint64_t bits) { return (int)((bits >> 52) & 0x7FFu); }

// round(v * 2^s) for the double with bit pattern `bits`, rounding half away from zero.
// Requires |v| * 2^s < 2^62. Zero and subnormal inputs give 0 (callers treat an exponent
// field of 0x7FF separately).
__device__ __forceinline__ long long f64_to_fixed(uint64_t bits, int s) {
  const int e = f64_exponent_field(bits);
  const uint64_t M = (bits & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  const int k = e - 1075 + s;  // v = M * 2^(e - 1075)
  uint64_t mag;
  if (k >= 0) {
    mag = M << (k > 10 ? 10 : k);
  } else {
    const int r = -k;  // >= 1
    const uint64_t t = M >> (r - 1 > 63 ? 63 : r - 1);
    mag = (t + 1) >> 1;
  }
  mag = (e == 0) ? 0ull : mag;
  const long long v = (long long)mag;
  return (bits >> 63) ? -v : v;
}

// W * 2^scale as a double, correctly rounded (to nearest, ties to even); results below the
// normal range flush to a signed zero. |W| <= 2^62.
__device__ __forceinline__ double fixed_to_f64(long long W, int scale) {
  const uint64_t sign = (uint64_t)W & 0x8000000000000000ull;
  const uint64_t mag = W < 0 ? (uint64_t)(-W) : (uint64_t)W;
  const int lz = __clzll((long long)mag);  // 64 when mag == 0
  const uint64_t m = mag << (lz & 63);      // leading one at bit 63
  uint64_t mant = m >> 11;
  const uint64_t rem = m & 0x7FFull;
  mant += (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ? 1ull : 0ull;
  int e = 63 - lz + scale + 1023;
  if (mant >> 53) {
    mant >>= 1;
    e += 1;
  }
  uint64_t bits = sign | ((uint64_t)e << 52) | (mant & 0x000FFFFFFFFFFFFFull);
  bits = (mag == 0 || e <= 0) ? sign : bits;
  bits = (e >= 0x7FF) ? (sign | 0x7FF0000000000000ull) : bits;
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double f64_nan() { return __longlong_as_double(0x7FF8000000000000ll); }
__device__ __forceinline__ float f32_nan() { return __int_as_float(0x7FC00000); }

// ------------------------------------------------------- TwoSum (Knuth), FP32 -- exact split --
// s + e == a + b exactly, s = fl(a + b). No multiplications, so no contraction applies.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

}  // namespace pauli

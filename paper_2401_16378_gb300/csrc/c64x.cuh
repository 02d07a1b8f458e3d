// c64x.cuh -- compensated FP32 arithmetic of the two-stage complex64 decomposition.
//
// Each real value is an unevaluated sum hi + lo of two floats. The high part lives on a
// power-of-two grid q chosen per XY-mask (per tile in stage 1, per mask in stage 2) from the
// mask's largest exponent so that every sum the remaining butterfly stages form stays below
// 2^24 q: all high-part additions are exact, so their TwoSum error term is identically zero and is
// not computed. The low parts carry the compensation and are added in plain FP32.
//  - split (error-free): with the anchor C = 1.5 * 2^23 * q, hi = fl(x + C) - C rounds x to the
//    grid and lo = x - hi is exact; (C, x) -> (hi, lo) is Fast2Sum with |C| > |x|, the
//    ExtractScalar step of Rump, Ogita and Oishi's accurate summation (SIAM J. Sci. Comput. 31(1),
//    2008).
//  - stage 1 (6 stages over the tile's rows): q1 = 2^(6 - 24) M1, M1 = 2^(E1 - 126) > every |x| of
//    the mask in the tile (E1: its largest float exponent field).
//  - between the stages each stage-1 value is kept as one float per part, fl(hi + lo) (the
//    scratch ring then holds 8 bytes per value, as G does).
//  - stage 2 (the other N - 6 stages): each stored value is split again, on the mask's grid
//    q2 = 2^(N + 1 - 24) Mm (Mm from the largest exponent over all tiles; one bit of headroom
//    for the rounding of the tiles' sums): hi2 = fl(x + C2) - C2, lo2 = x - hi2, exact.
//  - output: fl(hi + lo) times the exact 2^-N, times i^k.
// Error: the high parts are exact; the low parts start below q2 / 2 and FP32 recursive summation of
// 2^N of them errs by at most about N 2^-24 2^N q2 / 2 = N 2^(2N - 48) Mm in a sum, i.e. N 2^(N - 48) Mm
// in a coefficient (about 8e-10 Mm at N = 14). The rounding of the stage-1 values adds at most
// 2^-24 of each (|x| <= 2^6 Mm) to 2^(N - 6) terms of a sum: 2^-24 Mm in a coefficient in the
// worst case, of the order of the final rounding of a coefficient to FP32, and much less for
// values of mixed signs (the errors of independent tiles average out).
// Inputs of magnitude above about 2^(126 - N) would leave the FP32 range in the sums: the anchor of
// such a mask is NaN, so all of its outputs are NaN.
#pragma once
#include "xordiag_impl.cuh"

namespace pauli {
namespace xd {

// The split, the butterflies and the output of ArC64 (xordiag_impl.cuh); what differs is the grid:
// growth 2^6 over the stage-1 tile, then growth 2^(N + 1) over the whole mask, onto which stage 2
// re-splits the high parts (regrid).
struct ArC64X : ArC64 {
  static constexpr bool kRegrid = true;  // stage 2 re-splits the tiles on the mask's grid
  // out_scale == 0: stage 1 (6 butterfly stages); out_scale < 0: stage 2 (growth 2^(N + 1) in all),
  // with the output scale 2^out_scale
  __device__ static __forceinline__ Conv make_conv(int N, uint32_t Ekey, int out_scale) {
    return Conv{anchor(Ekey >> 23, out_scale == 0 ? 6 : N + 1), __int_as_float((127 + out_scale) << 23)};
  }
  // A stage-1 value as the scratch keeps it: each part's pair (hi, lo) rounded once to a float.
  __device__ static __forceinline__ uint2 pack_rounded(const Elem& a) {
    return make_uint2(__float_as_uint(__fadd_rn(a.rh, a.rl)), __float_as_uint(__fadd_rn(a.ih, a.il)));
  }
  __device__ static __forceinline__ Elem unpack_rounded(const uint2& q) {
    return Elem{__uint_as_float(q.x), 0.0f, __uint_as_float(q.y), 0.0f};
  }
  // re-split a stage-1 value x = hi + lo on the mask's stage-2 grid: hi2 = fl(hi + C2) - C2 and
  // hi - hi2 are exact (the split above)
  __device__ static __forceinline__ void regrid(Elem& a, const Conv& cv) {
    float h, r;
    h = __fsub_rn(__fadd_rn(a.rh, cv.anchor), cv.anchor);
    r = __fsub_rn(a.rh, h);
    a.rh = h;
    a.rl = __fadd_rn(a.rl, r);
    h = __fsub_rn(__fadd_rn(a.ih, cv.anchor), cv.anchor);
    r = __fsub_rn(a.ih, h);
    a.ih = h;
    a.il = __fadd_rn(a.il, r);
  }
};

// Real-part output: Re(v i^k) = (-1)^[k in {1, 2}] (k odd ? Im v : Re v), times the scale.
template <>
struct ReOut<ArC64X> : ArC64X {
  __device__ static __forceinline__ void store_hint(void* p, unsigned long long i, const Elem& a, const Conv& cv,
                                                    uint32_t k, uint64_t pol) {
    const float v = (k & 1u) ? __fadd_rn(a.ih, a.il) : __fadd_rn(a.rh, a.rl);
    const float o = __fmul_rn(((k ^ (k >> 1)) & 1u) ? -v : v, cv.scale);
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(reinterpret_cast<float*>(p) + i), "f"(o), "l"(pol)
                 : "memory");
  }
};

}  // namespace xd
}  // namespace pauli

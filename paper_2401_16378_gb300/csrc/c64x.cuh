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
//  - stage 2 (the other N - 6 stages): the high parts of every tile are re-split on the mask's
//    grid q2 = 2^(N + 1 - 24) Mm (Mm from the largest exponent over all tiles; one bit of headroom
//    for the re-rounding of the tiles' sums): hi2 = fl(hi + C2) - C2, lo2 = lo + (hi - hi2), where
//    hi - hi2 is exact (Sterbenz: hi2 is hi rounded to a coarser grid).
//  - output: fl(hi + lo) times the exact 2^-N, times i^k.
// Error: the high parts are exact; the low parts start below q2 / 2 and FP32 recursive summation of
// 2^N of them errs by at most about N 2^-24 2^N q2 / 2 = N 2^(2N - 48) Mm in a sum, i.e. N 2^(N - 48) Mm
// in a coefficient (about 8e-10 Mm at N = 14), below the final rounding of a coefficient to FP32.
// Inputs of magnitude above 2^(127 - N) overflow (the sums of 2^N of them leave the FP32 range).
#pragma once
#include "xordiag_impl.cuh"

namespace pauli {
namespace xd {

struct C64XConv {
  float anchor;  // 1.5 * 2^23 * grid
  float scale;   // output scale 2^out_scale (stage 2)
  bool nan;
};

struct ArC64X {
  using Raw = float2;
  using Elem = ArC64::Elem;  // (rh, rl, ih, il)
  using Conv = C64XConv;
  static constexpr bool kScaled = true;
  static constexpr bool kRegrid = true;  // stage 2 re-splits the tiles on the mask's grid
  __device__ static __forceinline__ Raw raw_unpack(const uint4& q) {
    return make_float2(__uint_as_float(q.x), __uint_as_float(q.y));
  }
  // largest exponent field of the two parts (compares as an integer)
  __device__ static __forceinline__ uint32_t exp_key(const Raw& r) {
    return max(__float_as_uint(r.x) & 0x7F800000u, __float_as_uint(r.y) & 0x7F800000u);
  }
  __device__ static __forceinline__ uint32_t key_exp(uint32_t key) { return key >> 23; }
  __device__ static __forceinline__ uint32_t exp_to_key(uint32_t e) { return e << 23; }
  // anchor for growth of 2^G over a mask whose largest exponent field is E:
  // C = 1.5 * 2^(E + G - 127), i.e. exponent field E + G, significand 1.5
  __device__ static __forceinline__ float anchor(uint32_t E, int G) {
    return __uint_as_float(((E + (uint32_t)G) << 23) | 0x00400000u);
  }
  // out_scale == 0: stage 1 (6 butterfly stages); out_scale < 0: stage 2 (growth 2^(N + 1) in all),
  // with the output scale 2^out_scale
  __device__ static __forceinline__ Conv make_conv(int N, uint32_t Ekey, int out_scale) {
    const uint32_t E = Ekey >> 23;
    Conv c;
    c.nan = E == 0xFFu || E + (uint32_t)N + 1u > 0xFEu;
    c.anchor = anchor(E, out_scale == 0 ? 6 : N + 1);
    c.scale = __int_as_float((127 + out_scale) << 23);
    return c;
  }
  __device__ static __forceinline__ void split(float x, float C, float& hi, float& lo) {
    hi = __fsub_rn(__fadd_rn(x, C), C);
    lo = __fsub_rn(x, hi);
  }
  template <int LPRE>
  __device__ static __forceinline__ Elem convert(const Raw& r, const Conv& cv, uint32_t) {
    Elem e;
    split(r.x, cv.anchor, e.rh, e.rl);
    split(r.y, cv.anchor, e.ih, e.il);
    return e;
  }
  __device__ static __forceinline__ void bfly(Elem& a, Elem& b) {
    const float rh0 = __fadd_rn(a.rh, b.rh), rh1 = __fsub_rn(a.rh, b.rh);
    const float rl0 = __fadd_rn(a.rl, b.rl), rl1 = __fsub_rn(a.rl, b.rl);
    const float ih0 = __fadd_rn(a.ih, b.ih), ih1 = __fsub_rn(a.ih, b.ih);
    const float il0 = __fadd_rn(a.il, b.il), il1 = __fsub_rn(a.il, b.il);
    a = Elem{rh0, rl0, ih0, il0};
    b = Elem{rh1, rl1, ih1, il1};
  }
  // re-split a stage-1 value on the mask's stage-2 grid
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
  __device__ static __forceinline__ uint4 pack(const Elem& a) { return ArC64::pack(a); }
  __device__ static __forceinline__ Elem unpack(const uint4& q) { return ArC64::unpack(q); }
  __device__ static __forceinline__ float2 out_value(const Elem& a, const Conv& cv, uint32_t k) {
    float re = __fadd_rn(a.rh, a.rl), im = __fadd_rn(a.ih, a.il);
    mul_i_pow(re, im, k);
    return make_float2(__fmul_rn(re, cv.scale), __fmul_rn(im, cv.scale));
  }
  __device__ static __forceinline__ void store_hint(void* p, unsigned long long i, const Elem& a, const Conv& cv,
                                                    uint32_t k, uint64_t pol) {
    const float2 o = out_value(a, cv, k);
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1,%2}, %3;" ::"l"(reinterpret_cast<float2*>(p) + i),
                 "f"(o.x), "f"(o.y), "l"(pol)
                 : "memory");
  }
  __device__ static __forceinline__ void align(Elem&, int) {}
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

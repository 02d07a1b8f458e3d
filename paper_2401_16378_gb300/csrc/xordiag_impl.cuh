// xordiag_impl.cuh -- building blocks of the XOR-diagonal kernels (see xordiag.cu): unit
// layouts, the shared-memory exchange, fixed-point conversions and arithmetic policies.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace pauli {
namespace xd {

// A unit holds 2^UB elements, 2^RB per thread in registers (RB = 4: 16 elements, RB = 3: 8):
//   (UB, RB) = (13, 4): 512 threads, one CTA per SM   (12, 4): 256 threads, two per SM
//              (12, 3): 512 threads, two CTAs per SM  (13, 3): 1024 threads, one per SM
// Fewer elements per thread mean fewer registers and more resident warps to hide latency, at
// the price of one more shared-memory exchange per unit.
template <int UB, int RB>
struct Unit {
  static constexpr int kThreads = 1 << (UB - RB);
  static constexpr int kMinBlocks = UB == 12 ? 2 : 1;
  static constexpr size_t kSmem = (size_t)16 << UB;
};

// Shared-memory slot swizzle: the low 3 bits of a 16-byte slot index are XORed with a
// linear function of its higher bits. The columns were chosen so that in every exchange
// of every layout below (both unit sizes, and the cluster combine) the 8 lanes of each
// quarter-warp touch 8 distinct bank groups.
__host__ __device__ constexpr uint32_t swz_col(int p) {
  return p == 3 ? 7u : p == 4 ? 4u : p == 5 ? 7u : p == 6 ? 5u : p == 7 ? 3u : p == 8 ? 6u : p == 9 ? 3u
       : p == 10 ? 1u : p == 11 ? 5u : p == 12 ? 5u : 0u;
}
__host__ __device__ constexpr uint32_t swz_term(uint32_t u) {
  uint32_t f = 0;
  for (int p = 3; p < 13; ++p)
    if ((u >> p) & 1u) f ^= swz_col(p);
  return f;
}
// 16-byte shared-memory accesses (one instruction each)
__device__ __forceinline__ void sts128(uint32_t addr, const uint4& v) {
  asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}
__device__ __forceinline__ uint4 lds128(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr) : "memory");
  return v;
}
__host__ __device__ constexpr uint32_t spread_c(uint32_t v) {
  uint32_t r = 0;
  for (int b = 0; b < 16; ++b) r |= ((v >> b) & 1u) << (2 * b);
  return r;
}

// Layout of a unit of 2^UB elements for L transformed row bits, K = UB - L class bits and RB
// register bits. Element index u = class | (row << K). The L row bits are cut into groups of
// at most RB bits: the top (possibly short) group first, then the others from bit 0 upwards,
// so the lowest output bits are transformed before the last phase and sit in the lanes when
// the unit is stored. Phase p transforms group p; its registers hold that group (padded with
// the lowest other row bits), its UB - RB thread-index bits hold the remaining u bits in
// ascending order, so lanes always vary the class bits first: coalesced sectors on load and
// store.
template <int UB, int L, int RB>
struct Layout {
  static constexpr int K = UB - L;
  static constexpr int E = 1 << RB;  // elements per thread
  static constexpr int TB = UB - RB;  // thread-index bits
  static constexpr int FULL = L / RB, REM = L % RB;
  static constexpr int NPH = FULL + (REM ? 1 : 0);
  __host__ __device__ static constexpr int gstart(int p) {
    return REM ? (p == 0 ? FULL * RB : (p - 1) * RB) : (p == 0 ? (FULL - 1) * RB : (p - 1) * RB);
  }
  __host__ __device__ static constexpr int gcount(int p) { return (REM && p == 0) ? REM : RB; }
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
    for (int k = 0; k < RB; ++k)
      if (regpos(p, k) == pos) return true;
    return false;
  }
  __host__ __device__ static constexpr int thrpos(int p, int k) {
    int need = k;
    for (int pos = 0; pos < UB; ++pos)
      if (!is_reg(p, pos)) {
        if (need == 0) return pos;
        --need;
      }
    return -1;
  }
  __host__ __device__ static constexpr uint32_t reg_u(int p, int j) {
    uint32_t u = 0;
    for (int k = 0; k < RB; ++k)
      if ((j >> k) & 1) u |= 1u << regpos(p, k);
    return u;
  }
  // register position k as a bit index of the row (or -1)
  __host__ __device__ static constexpr int regrow(int p, int k) { return k < RB ? regpos(p, k) - K : -1; }
  __device__ static __forceinline__ uint32_t thread_u(int p, uint32_t t) {
    uint32_t u = 0;
#pragma unroll
    for (int k = 0; k < TB; ++k) u |= ((t >> k) & 1u) << thrpos(p, k);
    return u;
  }
};

// ------------------------------------------------------- fixed point <-> FP64 (integer only) --
// Measured on GB300 (lanes/clk/SM): integer add ~110-128, logic/shift/select/IMAD ~64,
// int->float convert ~64, clz/popc ~16, FP64 ~2. The conversions below use adds where they can
// and no clz, popc or FP64 instruction on their common path.

// Per-class conversion state of the complex128 path.
struct FixConv {
  int rbase;      // right shift of the (pre-shifted) significand is rbase - exponent field
  int obias;      // biased FP64 exponent of 2^63 * output scale
  uint32_t oexp;  // (obias - 1 - 63 + 31 + 127 ... ) folded constant, see from_fixed
  bool slow;      // tiny class maximum (zeros and underflow need the general path), or NaN
  bool nan;       // class contains Inf or NaN: every output is NaN
};

// round-toward-zero(v * 2^s) of the double (hi, lo) as int64; LPRE = max(0, 9 - N) is a
// constant left pre-shift so that the remaining shift is always to the right. Zero and
// subnormal inputs give 0.
template <int LPRE>
__device__ __forceinline__ long long to_fixed(uint32_t hi, uint32_t lo, const FixConv& cv) {
  const int e = (int)((hi >> 20) & 0x7FFu);
  unsigned long long m = ((unsigned long long)((hi & 0x000FFFFFu) | 0x00100000u) << 32) | lo;
  if (LPRE > 0) m <<= LPRE;
  int r = cv.rbase - e;
  if (cv.slow) r = e ? r : 63;  // zero / subnormal (only reachable when rbase < 64)
  m >>= min(r, 63);             // significand < 2^55, so a shift by 63 gives 0
  const long long sg = (long long)((int)hi >> 31);
  return ((long long)m ^ sg) - sg;
}

// |W| * 2^(obias - 1086) rounded toward zero, with sign bit `sign` (bit 31), or NaN for a NaN
// class. The general path: zero, a small |W|, underflow.
static __device__ __noinline__ double from_fixed_small(unsigned long long a, uint32_t sign, int obias, bool nan) {
  if (nan) return f64_nan();
  if (a == 0ull) return __hiloint2double((int)sign, 0);
  const int lz = __clzll((long long)a);
  const unsigned long long m = a << lz;  // leading one at bit 63
  const int e = obias - lz;
  if (e <= 0) return __hiloint2double((int)sign, 0);  // below the normal range
  const uint32_t hi = (uint32_t)(m >> 43) + ((uint32_t)(e - 1) << 20);
  return __hiloint2double((int)(hi | sign), (int)(uint32_t)(m >> 11));
}
// Double nearest toward zero to W * 2^(obias - 1086), its sign bit XORed with negbit (0 or
// 1 << 31). |W| <= 2^62.
__device__ __forceinline__ double from_fixed(long long W, const FixConv& cv, uint32_t negbit) {
  const long long S = W >> 63;
  const unsigned long long a = (unsigned long long)((W ^ S) - S);
  const uint32_t sign = ((uint32_t)((unsigned long long)W >> 32) ^ negbit) & 0x80000000u;
  const uint32_t ah = (uint32_t)(a >> 32);
  if (ah == 0u || cv.slow) return from_fixed_small(a, sign, cv.obias, cv.nan);
  // floor(log2(ah)) from the exponent of an exact-toward-zero float conversion
  const uint32_t fe = __float_as_uint(__uint2float_rz(ah)) >> 23;  // 127 + floor(log2 ah)
  const unsigned long long m = a << (158u - fe);                    // leading one at bit 63
  // exponent field = obias - 158 + fe; the implicit one at bit 20 adds 1; the sign is the
  // top bit of a sum that stays below 2^31 without it
  const uint32_t hi = (uint32_t)(m >> 43) + (fe << 20) + (cv.oexp + sign);
  return __hiloint2double((int)hi, (int)(uint32_t)(m >> 11));
}

// popc(x & y) for a compile-time y with few bits: x's bits at those positions, pre-extracted
// into xb[] by the caller (xb[k] = bit pos_k of x), summed with integer adds instead of popc.
template <int P0, int P1, int P2, int P3>
struct BitSum {
  uint32_t b[4];
  __device__ __forceinline__ void init(uint32_t x) {
    b[0] = P0 >= 0 ? (x >> (P0 < 0 ? 0 : P0)) & 1u : 0u;
    b[1] = P1 >= 0 ? (x >> (P1 < 0 ? 0 : P1)) & 1u : 0u;
    b[2] = P2 >= 0 ? (x >> (P2 < 0 ? 0 : P2)) & 1u : 0u;
    b[3] = P3 >= 0 ? (x >> (P3 < 0 ? 0 : P3)) & 1u : 0u;
  }
  // sum over the set bits k of the 4-bit index j of b[k]
  __device__ __forceinline__ uint32_t at(int j) const {
    return ((j & 1) ? b[0] : 0u) + ((j & 2) ? b[1] : 0u) + ((j & 4) ? b[2] : 0u) + ((j & 8) ? b[3] : 0u);
  }
};

// ---------------------------------------------------------------------- arithmetic policies
struct ArC128 {
  using Raw = uint4;  // (re.lo, re.hi, im.lo, im.hi) bit patterns
  struct Elem {
    long long re, im;
  };
  using Conv = FixConv;
  static constexpr bool kScaled = true;
  // gathered rows are touched once: no L1 allocation (it would evict useful lines), and a
  // 128-byte L2 fetch so the neighbouring masks' sectors arrive with this one
  __device__ static __forceinline__ Raw load(const void* p, unsigned long long i) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::128B.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(reinterpret_cast<const uint4*>(p) + i));
    return v;
  }
  __device__ static __forceinline__ void prefetch(const void* p, unsigned long long i) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const uint4*>(p) + i));
  }
  // masked exponent fields (compare as integers)
  __device__ static __forceinline__ uint32_t exp_key(const Raw& r) { return max(r.y & 0x7FF00000u, r.w & 0x7FF00000u); }
  __device__ static __forceinline__ uint4 raw_pack(const Raw& r) { return r; }
  __device__ static __forceinline__ Raw raw_unpack(const uint4& q) { return q; }
  __device__ static __forceinline__ Conv make_conv(int N, uint32_t Ekey, int out_scale_exp) {
    // 2^N terms of magnitude < 2^(E-1022) * 2^s must stay below 2^62: s = 1084 - N - E.
    const int E = (int)(Ekey >> 20);
    Conv c;
    c.nan = E == 0x7FF;
    const int s = (E == 0 || c.nan) ? 0 : 1084 - N - E;
    const int lpre = N < 9 ? 9 - N : 0;
    c.rbase = 1075 - s + lpre;
    c.obias = 1086 + out_scale_exp - s;  // 1023 + 63 + scale
    c.oexp = (uint32_t)(c.obias - 158 - 1) << 20;
    c.slow = c.rbase < 64 || c.obias <= 64 || c.nan;
    return c;
  }
  // Converted element times i^k (k mod 4).
  template <int LPRE>
  __device__ static __forceinline__ Elem convert(const Raw& r, const Conv& cv, uint32_t k) {
    const bool swap = k & 1u;
    uint32_t ah = swap ? r.w : r.y, al = swap ? r.z : r.x;
    uint32_t bh = swap ? r.y : r.w, bl = swap ? r.x : r.z;
    ah ^= ((k ^ (k >> 1)) & 1u) << 31;  // i^k: re' = (-1)^[k in {1,2}] (k odd ? im : re)
    bh ^= ((k >> 1) & 1u) << 31;        //       im' = (-1)^[k in {2,3}] (k odd ? re : im)
    return Elem{to_fixed<LPRE>(ah, al, cv), to_fixed<LPRE>(bh, bl, cv)};
  }
  __device__ static __forceinline__ void bfly(Elem& a, Elem& b) {
    const long long r0 = a.re + b.re, r1 = a.re - b.re, i0 = a.im + b.im, i1 = a.im - b.im;
    a.re = r0;
    a.im = i0;
    b.re = r1;
    b.im = i1;
  }
  __device__ static __forceinline__ uint4 pack(const Elem& a) {
    return make_uint4((uint32_t)a.re, (uint32_t)((unsigned long long)a.re >> 32), (uint32_t)a.im,
                      (uint32_t)((unsigned long long)a.im >> 32));
  }
  __device__ static __forceinline__ Elem unpack(const uint4& q) {
    return Elem{(long long)(((unsigned long long)q.y << 32) | q.x), (long long)(((unsigned long long)q.w << 32) | q.z)};
  }
  // W * 2^scale * i^k as a double pair (NaN for a NaN class).
  __device__ static __forceinline__ double2 out_value(const Elem& a, const Conv& cv, uint32_t k) {
    const bool swap = k & 1u;
    const long long x = swap ? a.im : a.re, y = swap ? a.re : a.im;
    const uint32_t k31 = k << 31, k30 = k << 30;  // bits 0 and 1 of k at bit 31
    double2 o;
    o.x = from_fixed(x, cv, k31 ^ k30);  // negated for k = 1, 2
    o.y = from_fixed(y, cv, k30);         // negated for k = 2, 3
    return o;
  }
  __device__ static __forceinline__ void store(void* p, unsigned long long i, const Elem& a, const Conv& cv, uint32_t k) {
    reinterpret_cast<double2*>(p)[i] = out_value(a, cv, k);
  }
  __device__ static __forceinline__ void store_value(void* p, unsigned long long i, const double2& o) {
    reinterpret_cast<double2*>(p)[i] = o;
  }
  __device__ static __forceinline__ Raw conj(const Raw& r) { return make_uint4(r.x, r.y, r.z, r.w ^ 0x80000000u); }
  __device__ static __forceinline__ Raw real_part(const Raw& r) { return make_uint4(r.x, r.y, 0u, 0u); }
  // Loaded element times a real factor f (one FP64 rounding per part).
  __device__ static __forceinline__ Raw weigh(const Raw& r, double f) {
    const double re = __hiloint2double((int)r.y, (int)r.x) * f, im = __hiloint2double((int)r.w, (int)r.z) * f;
    return make_uint4((uint32_t)__double2loint(re), (uint32_t)__double2hiint(re), (uint32_t)__double2loint(im),
                      (uint32_t)__double2hiint(im));
  }
  // Same, with an L2 cache policy (createpolicy) for the store.
  __device__ static __forceinline__ void store_hint(void* p, unsigned long long i, const Elem& a, const Conv& cv,
                                                    uint32_t k, uint64_t pol) {
    const double2 o = out_value(a, cv, k);
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1,%2}, %3;" ::"l"(reinterpret_cast<double2*>(p) + i),
                 "d"(o.x), "d"(o.y), "l"(pol)
                 : "memory");
  }
  // Arithmetic right shift by sh in [0, 63]: re-expresses a value held at scale 2^s at 2^(s - sh).
  __device__ static __forceinline__ void align(Elem& a, int sh) {
    a.re >>= sh;
    a.im >>= sh;
  }
};

// complex64, compensated FP32 on a per-mask power-of-two grid. Each real value is an
// unevaluated sum hi + lo of two floats, split error-free on input: with the anchor
// C = 1.5 * 2^23 * q, hi = fl(x + C) - C rounds x to the grid q and lo = x - hi is exact (Fast2Sum
// with |C| > |x|; the ExtractScalar step of Rump, Ogita and Oishi, SIAM J. Sci. Comput. 31(1),
// 2008). q = 2^(N + 1 - 23) 2^(E - 127) for the mask's largest float exponent field E, so every sum
// of 2^N high parts stays below 2^24 q: all high-part additions are exact (their TwoSum error term
// is identically zero and is not computed), and the low parts, added in plain FP32, carry the
// compensation. Error before the final rounding: about N 2^(N - 47) 2^(E - 127) per coefficient.
// A mask whose anchor would leave the FP32 range (inputs above about 2^(126 - N)) or that holds
// a non-finite value gets a NaN anchor, so all its outputs are NaN.
struct C64Conv {
  float anchor;  // 1.5 * 2^23 * grid
  float scale;   // output scale 2^out_scale, exact
};

struct ArC64 {
  using Raw = float2;
  struct Elem {
    float rh, rl, ih, il;
  };
  using Conv = C64Conv;
  static constexpr bool kScaled = true;
  __device__ static __forceinline__ Raw load(const void* p, unsigned long long i) {
    float2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::128B.v2.f32 {%0,%1}, [%2];"
                 : "=f"(v.x), "=f"(v.y)
                 : "l"(reinterpret_cast<const float2*>(p) + i));
    return v;
  }
  __device__ static __forceinline__ void prefetch(const void* p, unsigned long long i) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const float2*>(p) + i));
  }
  // largest exponent field of the two parts (compares as an integer)
  __device__ static __forceinline__ uint32_t exp_key(const Raw& r) {
    return max(__float_as_uint(r.x) & 0x7F800000u, __float_as_uint(r.y) & 0x7F800000u);
  }
  __device__ static __forceinline__ uint4 raw_pack(const Raw& r) { return make_uint4(__float_as_uint(r.x), __float_as_uint(r.y), 0u, 0u); }
  __device__ static __forceinline__ Raw raw_unpack(const uint4& q) { return make_float2(__uint_as_float(q.x), __uint_as_float(q.y)); }
  // anchor for a growth of 2^G over a mask whose largest exponent field is E: exponent field
  // E + G, significand 1.5; NaN when that leaves the finite range or E marks Inf / NaN
  __device__ static __forceinline__ float anchor(uint32_t E, int G) {
    const uint32_t e = E + (uint32_t)G;
    return __uint_as_float(E >= 0xFFu || e > 0xFEu ? 0x7FC00000u : (e << 23) | 0x00400000u);
  }
  __device__ static __forceinline__ Conv make_conv(int N, uint32_t Ekey, int out_scale_exp) {
    return Conv{anchor(Ekey >> 23, N + 1), __int_as_float((127 + out_scale_exp) << 23)};
  }
  __device__ static __forceinline__ void split(float x, float C, float& hi, float& lo) {
    hi = __fsub_rn(__fadd_rn(x, C), C);
    lo = __fsub_rn(x, hi);
  }
  // Converted element times i^k (k mod 4; exact).
  template <int LPRE>
  __device__ static __forceinline__ Elem convert(const Raw& r, const Conv& cv, uint32_t k) {
    float re = r.x, im = r.y;
    mul_i_pow(re, im, k);
    Elem e;
    split(re, cv.anchor, e.rh, e.rl);
    split(im, cv.anchor, e.ih, e.il);
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
  __device__ static __forceinline__ uint4 pack(const Elem& a) {
    return make_uint4(__float_as_uint(a.rh), __float_as_uint(a.rl), __float_as_uint(a.ih), __float_as_uint(a.il));
  }
  __device__ static __forceinline__ Elem unpack(const uint4& q) {
    return Elem{__uint_as_float(q.x), __uint_as_float(q.y), __uint_as_float(q.z), __uint_as_float(q.w)};
  }
  __device__ static __forceinline__ float2 out_value(const Elem& a, const Conv& cv, uint32_t k) {
    float re = __fadd_rn(a.rh, a.rl), im = __fadd_rn(a.ih, a.il);
    mul_i_pow(re, im, k);
    return make_float2(__fmul_rn(re, cv.scale), __fmul_rn(im, cv.scale));
  }
  __device__ static __forceinline__ void store(void* p, unsigned long long i, const Elem& a, const Conv& cv, uint32_t k) {
    reinterpret_cast<float2*>(p)[i] = out_value(a, cv, k);
  }
  __device__ static __forceinline__ void store_value(void* p, unsigned long long i, const float2& o) {
    reinterpret_cast<float2*>(p)[i] = o;
  }
  __device__ static __forceinline__ Raw weigh(const Raw& r, float f) { return make_float2(r.x * f, r.y * f); }
  __device__ static __forceinline__ Raw conj(const Raw& r) { return make_float2(r.x, -r.y); }
  __device__ static __forceinline__ Raw real_part(const Raw& r) { return make_float2(r.x, 0.f); }
  __device__ static __forceinline__ void store_hint(void* p, unsigned long long i, const Elem& a, const Conv& cv,
                                                    uint32_t k, uint64_t pol) {
    const float2 o = out_value(a, cv, k);
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1,%2}, %3;" ::"l"(reinterpret_cast<float2*>(p) + i),
                 "f"(o.x), "f"(o.y), "l"(pol)
                 : "memory");
  }
  __device__ static __forceinline__ void align(Elem&, int) {}
};

// complex64 with TwoSum-compensated butterflies (FP32 value + FP32 error term per part): the
// arithmetic of the block-tiled two-stage kernel, whose tiles have no common grid.
struct C64TConv {
  float scale;
};

struct ArC64T {
  using Raw = float2;
  struct Elem {
    float rh, rl, ih, il;
  };
  using Conv = C64TConv;
  static constexpr bool kScaled = false;
  __device__ static __forceinline__ Raw load(const void* p, unsigned long long i) {
    float2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::128B.v2.f32 {%0,%1}, [%2];"
                 : "=f"(v.x), "=f"(v.y)
                 : "l"(reinterpret_cast<const float2*>(p) + i));
    return v;
  }
  __device__ static __forceinline__ void prefetch(const void* p, unsigned long long i) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const float2*>(p) + i));
  }
  __device__ static __forceinline__ uint32_t exp_key(const Raw&) { return 0u; }
  __device__ static __forceinline__ uint4 raw_pack(const Raw& r) { return make_uint4(__float_as_uint(r.x), __float_as_uint(r.y), 0u, 0u); }
  __device__ static __forceinline__ Raw raw_unpack(const uint4& q) { return make_float2(__uint_as_float(q.x), __uint_as_float(q.y)); }
  __device__ static __forceinline__ Conv make_conv(int, uint32_t, int out_scale_exp) {
    return Conv{__int_as_float((127 + out_scale_exp) << 23)};  // 2^scale, exact
  }
  template <int LPRE>
  __device__ static __forceinline__ Elem convert(const Raw& r, const Conv&, uint32_t k) {
    float re = r.x, im = r.y;
    mul_i_pow(re, im, k);
    return Elem{re, 0.f, im, 0.f};
  }
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
  __device__ static __forceinline__ uint4 pack(const Elem& a) {
    return make_uint4(__float_as_uint(a.rh), __float_as_uint(a.rl), __float_as_uint(a.ih), __float_as_uint(a.il));
  }
  __device__ static __forceinline__ Elem unpack(const uint4& q) {
    return Elem{__uint_as_float(q.x), __uint_as_float(q.y), __uint_as_float(q.z), __uint_as_float(q.w)};
  }
  __device__ static __forceinline__ float2 out_value(const Elem& a, const Conv& cv, uint32_t k) {
    float re = __fadd_rn(a.rh, a.rl), im = __fadd_rn(a.ih, a.il);
    mul_i_pow(re, im, k);
    return make_float2(__fmul_rn(re, cv.scale), __fmul_rn(im, cv.scale));
  }
  __device__ static __forceinline__ void store(void* p, unsigned long long i, const Elem& a, const Conv& cv, uint32_t k) {
    reinterpret_cast<float2*>(p)[i] = out_value(a, cv, k);
  }
  __device__ static __forceinline__ void store_value(void* p, unsigned long long i, const float2& o) {
    reinterpret_cast<float2*>(p)[i] = o;
  }
  __device__ static __forceinline__ Raw weigh(const Raw& r, float f) { return make_float2(r.x * f, r.y * f); }
  __device__ static __forceinline__ Raw conj(const Raw& r) { return make_float2(r.x, -r.y); }
  __device__ static __forceinline__ Raw real_part(const Raw& r) { return make_float2(r.x, 0.f); }
  __device__ static __forceinline__ void store_hint(void* p, unsigned long long i, const Elem& a, const Conv& cv,
                                                    uint32_t k, uint64_t pol) {
    const float2 o = out_value(a, cv, k);
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1,%2}, %3;" ::"l"(reinterpret_cast<float2*>(p) + i),
                 "f"(o.x), "f"(o.y), "l"(pol)
                 : "memory");
  }
  __device__ static __forceinline__ void align(Elem&, int) {}
};

// Real-part output: the arithmetic of Base, but only Re(v * i^k) is converted and stored,
// into an array of reals (double or float) indexed like the complex output. For a Hermitian
// G every c_n is real and this is all of it; for any G it is c_n((G + G^H) / 2).
// Re(v i^k) = (-1)^[k in {1, 2}] (k odd ? Im v : Re v).
template <class Base>
struct ReOut;

template <>
struct ReOut<ArC128> : ArC128 {
  __device__ static __forceinline__ double re_value(const Elem& a, const Conv& cv, uint32_t k) {
    return from_fixed((k & 1u) ? a.im : a.re, cv, (k << 31) ^ (k << 30));
  }
  __device__ static __forceinline__ void store(void* p, unsigned long long i, const Elem& a, const Conv& cv, uint32_t k) {
    reinterpret_cast<double*>(p)[i] = re_value(a, cv, k);
  }
  __device__ static __forceinline__ void store_hint(void* p, unsigned long long i, const Elem& a, const Conv& cv,
                                                    uint32_t k, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(reinterpret_cast<double*>(p) + i),
                 "d"(re_value(a, cv, k)), "l"(pol)
                 : "memory");
  }
};

template <>
struct ReOut<ArC64> : ArC64 {
  __device__ static __forceinline__ float re_value(const Elem& a, const Conv& cv, uint32_t k) {
    const float v = (k & 1u) ? __fadd_rn(a.ih, a.il) : __fadd_rn(a.rh, a.rl);
    return __fmul_rn(((k ^ (k >> 1)) & 1u) ? -v : v, cv.scale);
  }
  __device__ static __forceinline__ void store(void* p, unsigned long long i, const Elem& a, const Conv& cv, uint32_t k) {
    reinterpret_cast<float*>(p)[i] = re_value(a, cv, k);
  }
  __device__ static __forceinline__ void store_hint(void* p, unsigned long long i, const Elem& a, const Conv& cv,
                                                    uint32_t k, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(reinterpret_cast<float*>(p) + i),
                 "f"(re_value(a, cv, k)), "l"(pol)
                 : "memory");
  }
};

template <>
struct ReOut<ArC64T> : ArC64T {
  __device__ static __forceinline__ float re_value(const Elem& a, const Conv& cv, uint32_t k) {
    const float v = (k & 1u) ? __fadd_rn(a.ih, a.il) : __fadd_rn(a.rh, a.rl);
    return __fmul_rn(((k ^ (k >> 1)) & 1u) ? -v : v, cv.scale);
  }
  __device__ static __forceinline__ void store(void* p, unsigned long long i, const Elem& a, const Conv& cv, uint32_t k) {
    reinterpret_cast<float*>(p)[i] = re_value(a, cv, k);
  }
  __device__ static __forceinline__ void store_hint(void* p, unsigned long long i, const Elem& a, const Conv& cv,
                                                    uint32_t k, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(reinterpret_cast<float*>(p) + i),
                 "f"(re_value(a, cv, k)), "l"(pol)
                 : "memory");
  }
};

// Butterflies over the low G register-index bits.
template <class AR, int G, int E>
__device__ __forceinline__ void wht_regs(typename AR::Elem (&v)[E]) {
#pragma unroll
  for (int b = 0; b < G; ++b)
#pragma unroll
    for (int j = 0; j < E; ++j)
      if (!((j >> b) & 1)) AR::bfly(v[j], v[j | (1 << b)]);
}

// Barrier over the threads that hold a unit: the whole CTA, or (NamedSync) the first
// THREADS threads on hardware barrier ID (warp-specialised kernels).
struct CtaSync {
  __device__ static __forceinline__ void sync() { __syncthreads(); }
};
template <int ID, int THREADS>
struct NamedSync {
  __device__ static __forceinline__ void sync() { asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(THREADS) : "memory"); }
};

// Re-distribute the unit between threads from phase P's layout to phase P+1's, through shared
// memory: 16-byte slots, slot(u) = u ^ swz(u) (XOR-linear, so thread part and register part
// combine with one XOR; the base address is added afterwards).
template <class LY, class AR, int P, class SY = CtaSync>
__device__ __forceinline__ void exchange(typename AR::Elem (&v)[LY::E], uint32_t xaddr, uint32_t t) {
  SY::sync();
  const uint32_t ut = LY::thread_u(P, t);
  const uint32_t ft = ut ^ swz_term(ut);
#pragma unroll
  for (int j = 0; j < LY::E; ++j)
    sts128(xaddr + 16u * (ft ^ (LY::reg_u(P, j) ^ swz_term(LY::reg_u(P, j)))), AR::pack(v[j]));
  SY::sync();
  const uint32_t un = LY::thread_u(P + 1, t);
  const uint32_t fn = un ^ swz_term(un);
#pragma unroll
  for (int j = 0; j < LY::E; ++j)
    v[j] = AR::unpack(lds128(xaddr + 16u * (fn ^ (LY::reg_u(P + 1, j) ^ swz_term(LY::reg_u(P + 1, j))))));
}

// All phases of the local transform: butterflies, exchange, butterflies, ...
template <class LY, class AR, int P = 0, class SY = CtaSync>
__device__ __forceinline__ void local_wht(typename AR::Elem (&v)[LY::E], uint32_t xaddr, uint32_t t) {
  wht_regs<AR, LY::gcount(P), LY::E>(v);
  if constexpr (P + 1 < LY::NPH) {
    exchange<LY, AR, P, SY>(v, xaddr, t);
    local_wht<LY, AR, P + 1, SY>(v, xaddr, t);
  }
}

// Global element index of (class x, index y = y_t | y_j) where the thread part y_t and the
// register part y_j have disjoint bits:
//   MATRIX: G[y, y ^ x] = y_t*D + (y_t ^ x) + y_j*D ^ y_j (per-element: one add, one xor)
//   COEFFS: c[n(x, y)]  = n(x, y_t) ^ 3*spread(y_j)   (n(x, z): even bits x^z, odd bits z)
template <int N, bool MATRIX>
struct Addr {
  unsigned long long tb;  // thread part
  uint32_t q;             // y_t ^ x (matrix case)
  __device__ __forceinline__ void init(unsigned long long base, uint32_t x, uint32_t yt) {
    if (MATRIX) {
      tb = base + (unsigned long long)yt * (1ull << N);
      q = yt ^ x;
    } else {
      tb = base + pauli_index(x, yt);
      q = 0;
    }
  }
  __device__ __forceinline__ unsigned long long at(uint32_t yj) const {
    if (MATRIX) return tb + ((unsigned long long)yj << N) + (q ^ yj);
    return tb ^ (unsigned long long)(3u * spread_c(yj));
  }
};


// ------------------------------------------------- fused work at the two ends of a unit --
// Arguments of the fused forms (kernel parameters; unused by NoEpi).
struct EpiArgs {
  const void* w;     // 4^N real weights: double (complex128) or float (complex64)
  const void* g;     // one real scaling the weights (compose), or nullptr for 1
  double* partial;   // one partial loss per work unit (decompose)
};
// Plain decomposition / composition.
struct NoEpi {
  static constexpr bool kWeightIn = false, kNormOut = false, kMirror = false;
};
// Composition of weighted coefficients: each loaded c_n is multiplied by g w_n first.
struct WeightInEpi {
  static constexpr bool kWeightIn = true, kNormOut = false, kMirror = false;
};
// Decomposition that also accumulates sum_n w_n |c_n|^2 over the coefficients it stores.
struct NormOutEpi {
  static constexpr bool kWeightIn = false, kNormOut = true, kMirror = false;
};
// Decomposition of a Hermitian G from its upper triangle: an element G[r, r ^ x] below the
// diagonal (bit h of r set, h the top set bit of x) is read as conj(G[r ^ x, r]).
struct MirrorUpperEpi {
  static constexpr bool kWeightIn = false, kNormOut = false, kMirror = true;
};

// Per-thread accumulator of w_n |c_n|^2: FP64 for complex128; for complex64 a TwoSum-compensated
// FP32 pair, read out in FP64.
template <class AR>
struct NormAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(const double2& o, double w) { s = fma(w, fma(o.y, o.y, o.x * o.x), s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct NormAcc<ArC64> {
  float s = 0.f, e = 0.f;
  __device__ __forceinline__ void add(const float2& o, float w) {
    const float x = w * fmaf(o.y, o.y, o.x * o.x);
    const float t = s + x, bp = t - s;
    e += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)e; }
};
template <class AR>
struct RealOf {
  using T = double;
};
template <>
struct RealOf<ArC64> {
  using T = float;
};

// ------------------------------------------------------------- one single-CTA work unit --
// Classes [xb, xb + 2^K) of the N-qubit matrix whose elements start at index `base` of in/out
// (decompose: in = G, out = c; compose: in = c, out = G). smax holds 2^K words. prefetch()
// is called once the unit's own loads are in flight.
// EPI adds the fused work of WeightInEpi (compose) or NormOutEpi (decompose; the return value is
// then this thread's share of the unit's partial loss, else 0).
template <int UB, int RB, int N, class AR, bool COMPOSE, class Prefetch, class EPI = NoEpi>
__device__ __forceinline__ double run_unit(const void* __restrict__ in, void* __restrict__ out,
                                           unsigned long long base, uint32_t xb, int scale_exp, uint32_t xaddr,
                                           uint32_t* smax, uint32_t t, Prefetch prefetch,
                                           const EpiArgs& ea = EpiArgs{nullptr, nullptr, nullptr}) {
  using Real = typename RealOf<AR>::T;
  constexpr unsigned long long kNMask = (1ull << (2 * N)) - 1ull;
  using LY = Layout<UB, N, RB>;
  constexpr int K = LY::K;
  constexpr int E = LY::E;
  constexpr int LAST = LY::NPH - 1;
  constexpr int LPRE = N < 9 ? 9 - N : 0;
  const uint32_t c = t & ((1u << K) - 1u);  // class bits are the lowest thread bits in every phase
  const uint32_t x = xb | c;
  const uint32_t y0 = LY::thread_u(0, t) >> K;  // thread part of the load-phase index
  const uint32_t yl = LY::thread_u(LAST, t) >> K;
  const int out_scale = COMPOSE ? scale_exp : -N;
  Addr<N, !COMPOSE> ain;
  ain.init(base, x, y0);
  typename AR::Raw raw[E];
  uint32_t emax = 0;
  if constexpr (EPI::kMirror) {
    static_assert(!COMPOSE, "mirrored reads are for the decomposition");
    const uint32_t h = x ? 31u - (uint32_t)__clz(x) : 32u;
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const uint32_t r = y0 | (LY::reg_u(0, j) >> K);
      const bool lower = h < 32u && ((r >> h) & 1u);
      const unsigned long long i =
          lower ? base + ((unsigned long long)(r ^ x) << N) + r : ain.at(LY::reg_u(0, j) >> K);
      raw[j] = AR::load(in, i);
      if (lower) raw[j] = AR::conj(raw[j]);
      if (x == 0u) raw[j] = AR::real_part(raw[j]);  // the diagonal: its imaginary parts are not used
    }
  } else {
#pragma unroll
    for (int j = 0; j < E; ++j) raw[j] = AR::load(in, ain.at(LY::reg_u(0, j) >> K));
  }
  if constexpr (EPI::kWeightIn) {
    const Real* w = static_cast<const Real*>(ea.w);
    const Real g = ea.g ? *static_cast<const Real*>(ea.g) : Real(1);
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const Real wn = w[ain.at(LY::reg_u(0, j) >> K) & kNMask];
      raw[j] = AR::weigh(raw[j], g == Real(1) ? wn : g * wn);
    }
  }
#pragma unroll
  for (int j = 0; j < E; ++j) emax = max(emax, AR::exp_key(raw[j]));
  prefetch();
  uint32_t Ekey = 0;
  if constexpr (AR::kScaled) {
    if (t < (1u << K)) smax[t] = 0;
    __syncthreads();
#pragma unroll
    for (int m = 1 << K; m < 32; m <<= 1) emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, m));
    if (((t & 31u) >> K) == 0) atomicMax(&smax[c], emax);
    __syncthreads();
    Ekey = smax[c];
  }
  const typename AR::Conv cv = AR::make_conv(N, Ekey, out_scale);
  typename AR::Elem v[E];
  {
    // compose: times (-i)^popc(x&z) = i^(3 popc(x&z)), z = y0 | (register part)
    BitSum<LY::regrow(0, 0), LY::regrow(0, 1), LY::regrow(0, 2), LY::regrow(0, 3)> xb;
    xb.init(x);
    const uint32_t kt = COMPOSE ? (uint32_t)__popc(x & y0) : 0u;
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = AR::template convert<LPRE>(raw[j], cv, COMPOSE ? 3u * (kt + xb.at(j)) : 0u);
  }
  local_wht<LY, AR>(v, xaddr, t);
  Addr<N, COMPOSE> ao;
  ao.init(base, x, yl);
  // decompose: times i^popc(x&z), z = yl | (register part)
  BitSum<LY::regrow(LAST, 0), LY::regrow(LAST, 1), LY::regrow(LAST, 2), LY::regrow(LAST, 3)> xo;
  xo.init(x);
  const uint32_t ko = COMPOSE ? 0u : (uint32_t)__popc(x & yl);
  if constexpr (EPI::kNormOut) {
    const Real* w = static_cast<const Real*>(ea.w);
    NormAcc<AR> acc;
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const unsigned long long i = ao.at(LY::reg_u(LAST, j) >> K);
      const auto o = AR::out_value(v[j], cv, ko + xo.at(j));
      AR::store_value(out, i, o);
      acc.add(o, w[i & kNMask]);
    }
    return acc.value();
  } else {
#pragma unroll
    for (int j = 0; j < E; ++j)
      AR::store(out, ao.at(LY::reg_u(LAST, j) >> K), v[j], cv, COMPOSE ? 0u : ko + xo.at(j));
    return 0.0;
  }
}

// L2 prefetch of the elements run_unit will load for classes [xb, xb + 2^K).
template <int UB, int RB, int N, class AR, bool COMPOSE>
__device__ __forceinline__ void unit_prefetch(const void* in, unsigned long long base, uint32_t xb, uint32_t t) {
  using LY = Layout<UB, N, RB>;
  constexpr int K = LY::K;
  Addr<N, !COMPOSE> an;
  an.init(base, xb | (t & ((1u << K) - 1u)), LY::thread_u(0, t) >> K);
#pragma unroll
  for (int j = 0; j < LY::E; ++j) AR::prefetch(in, an.at(LY::reg_u(0, j) >> K));
}

// ----------------------------------------------- Hermitian G from its upper triangle --
// For a Hermitian G the XOR-diagonal of a class x != 0 satisfies e_x[r ^ x] = conj(e_x[r]).
// With h the top set bit of x, pair each row r having r_h = 0 with r ^ x (which has bit h set;
// r < r ^ x, so e_x[r] = G[r, r ^ x] lies above the diagonal). Then for every z
//   W_x[z] = sum_{r_h = 0} (-1)^popc(r & z) (e_x[r] + (-1)^popc(x & z) conj(e_x[r])),
// and with V[z'] the WHT over the N - 1 bits other than h of e_x restricted to r_h = 0
// (z' = z without bit h) this gives, for both z with that z',
//   c(x, z) = 2^-N i^popc(x&z) W_x[z] = 2^(1-N) Re(V[z'] i^popc(x&z)).
// So a unit reads only the upper triangle (half of G), transforms 2^(N-1) rows per class with
// the same machinery, and each transformed value gives two real coefficients: z0 (z_h = 0)
// and z1 = z0 | 2^h, whose phases differ by one factor i. The classes [xb, xb + 2^K) of a unit
// must share their top bit: xb >= 2^K. AR stores real parts (ReOut<...>).
template <int UB, int RB, int N, class AR, class Prefetch>
__device__ __forceinline__ void run_unit_herm(const void* __restrict__ in, void* __restrict__ out,
                                              unsigned long long base, uint32_t xb, uint32_t xaddr, uint32_t* smax,
                                              uint32_t t, Prefetch prefetch) {
  constexpr int NH = N - 1;  // transformed row bits
  using LY = Layout<UB, NH, RB>;
  constexpr int K = LY::K;
  constexpr int E = LY::E;
  constexpr int LAST = LY::NPH - 1;
  constexpr int LPRE = N < 9 ? 9 - N : 0;
  const uint32_t c = t & ((1u << K) - 1u);
  const uint32_t x = xb | c;
  const uint32_t h = 31u - (uint32_t)__clz(xb);  // top bit of every class of the unit
  const uint32_t lowm = (1u << h) - 1u;
  // insert a zero at bit h: r' (N - 1 bits) -> r
  auto ins = [&](uint32_t v) { return (v & lowm) | ((v & ~lowm) << 1); };
  const uint32_t y0 = LY::thread_u(0, t) >> K;
  const uint32_t yl = LY::thread_u(LAST, t) >> K;
  const uint32_t r0 = ins(y0);
  typename AR::Raw raw[E];
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const uint32_t r = r0 | ins(LY::reg_u(0, j) >> K);
    raw[j] = AR::load(in, base + ((unsigned long long)r << N) + (r ^ x));
  }
  prefetch();
  uint32_t emax = 0;
#pragma unroll
  for (int j = 0; j < E; ++j) emax = max(emax, AR::exp_key(raw[j]));
  uint32_t Ekey = 0;
  if constexpr (AR::kScaled) {
    if (t < (1u << K)) smax[t] = 0;
    __syncthreads();
#pragma unroll
    for (int m = 1 << K; m < 32; m <<= 1) emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, m));
    if (((t & 31u) >> K) == 0) atomicMax(&smax[c], emax);
    __syncthreads();
    Ekey = smax[c];
  }
  // the class maximum over half the rows is the class maximum (the other half are conjugates)
  const typename AR::Conv cv = AR::make_conv(N, Ekey, 1 - N);
  typename AR::Elem v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = AR::template convert<LPRE>(raw[j], cv, 0u);
  local_wht<LY, AR>(v, xaddr, t);
  // outputs: z0 = ins(z'), z' = yl | (register part); n(x, z) = spread(x) ^ 3 spread(z) is
  // linear in z, and inserting bit h moves the spread bits at and above 2h up by two
  const uint32_t xc = (x & lowm) | ((x >> 1) & ~lowm);  // x without bit h, for popc(x & z0)
  const uint32_t sm = spread_c(0xFFFFu) & ((1u << (2 * h)) - 1u);
  auto ins3s = [&](uint32_t sp) { return 3u * ((sp & sm) | ((sp & ~sm) << 2)); };
  const unsigned long long tb = base + (unsigned long long)(spread16(x) ^ ins3s(spread16(yl)));
  const uint32_t flip = 3u << (2 * h);
  BitSum<LY::regrow(LAST, 0), LY::regrow(LAST, 1), LY::regrow(LAST, 2), LY::regrow(LAST, 3)> xo;
  xo.init(xc);
  const uint32_t ko = (uint32_t)__popc(xc & yl);
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const unsigned long long n0 = tb ^ ins3s(spread_c(LY::reg_u(LAST, j) >> K));
    const uint32_t k0 = ko + xo.at(j);
    AR::store(out, n0, v[j], cv, k0);
    AR::store(out, n0 ^ flip, v[j], cv, k0 + 1u);
  }
}

template <int UB, int RB, int N, class AR>
__device__ __forceinline__ void herm_prefetch(const void* in, unsigned long long base, uint32_t xb, uint32_t t) {
  using LY = Layout<UB, N - 1, RB>;
  constexpr int K = LY::K;
  const uint32_t x = xb | (t & ((1u << K) - 1u));
  const uint32_t lowm = (1u << (31u - (uint32_t)__clz(xb))) - 1u;
  auto ins = [&](uint32_t v) { return (v & lowm) | ((v & ~lowm) << 1); };
  const uint32_t r0 = ins(LY::thread_u(0, t) >> K);
#pragma unroll
  for (int j = 0; j < LY::E; ++j) {
    const uint32_t r = r0 | ins(LY::reg_u(0, j) >> K);
    AR::prefetch(in, base + ((unsigned long long)r << N) + (r ^ x));
  }
}

}  // namespace xd
}  // namespace pauli

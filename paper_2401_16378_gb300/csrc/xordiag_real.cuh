// xordiag_real.cuh -- arithmetic policy for real input matrices (float64), used with the
// XOR-diagonal kernels of xordiag_kernels.cuh and tiled_impl.cuh (xordiag_real.cu,
// tiled_real_r4.cu).
#pragma once
#include "xordiag_impl.cuh"

namespace pauli {
namespace xd {

// Real input (a float64 matrix): the arithmetic of ArC128 with zero imaginary parts, reading 8
// bytes per element. For real G the transform W_x[z] is real, so c(x, z) = 2^-N i^k W_x[z]
// (k = popc(x & z), the number of Y factors) is real for even k and imaginary for odd k; the
// output stores the real number a = c (-i)^(k mod 2) = (-1)^floor(k/2) 2^-N W_x[z].
struct ArR128 : ArC128 {
  using Raw = uint2;  // the double's bits (lo, hi)
  __device__ static __forceinline__ Raw load(const void* p, unsigned long long i) {
    uint2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::128B.v2.u32 {%0,%1}, [%2];"
                 : "=r"(v.x), "=r"(v.y)
                 : "l"(reinterpret_cast<const uint2*>(p) + i));
    return v;
  }
  __device__ static __forceinline__ void prefetch(const void* p, unsigned long long i) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const uint2*>(p) + i));
  }
  __device__ static __forceinline__ uint32_t exp_key(const Raw& r) { return r.y & 0x7FF00000u; }
  __device__ static __forceinline__ uint4 raw_pack(const Raw& r) { return make_uint4(r.x, r.y, 0u, 0u); }
  __device__ static __forceinline__ Raw raw_unpack(const uint4& q) { return make_uint2(q.x, q.y); }
  template <int LPRE>
  __device__ static __forceinline__ Elem convert(const Raw& r, const Conv& cv, uint32_t) {
    return Elem{to_fixed<LPRE>(r.y, r.x, cv), 0};
  }
  __device__ static __forceinline__ double real_value(const Elem& a, const Conv& cv, uint32_t k) {
    return from_fixed(a.re, cv, ((k >> 1) & 1u) << 31);
  }
  __device__ static __forceinline__ void store(void* p, unsigned long long i, const Elem& a, const Conv& cv, uint32_t k) {
    reinterpret_cast<double*>(p)[i] = real_value(a, cv, k);
  }
  __device__ static __forceinline__ void store_hint(void* p, unsigned long long i, const Elem& a, const Conv& cv,
                                                    uint32_t k, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(reinterpret_cast<double*>(p) + i),
                 "d"(real_value(a, cv, k)), "l"(pol)
                 : "memory");
  }
};

}  // namespace xd
}  // namespace pauli

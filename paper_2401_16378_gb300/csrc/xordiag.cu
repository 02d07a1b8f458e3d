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
// Work unit (single-pass kernels): 8192 elements, 16 per thread of a 512-thread CTA (or 4096
// on 256 threads, or 8 per thread on twice the threads), held in registers. For N <= 12 a
// unit is 2^K consecutive XY-masks (the "classes", K = 13 - N) times all 2^N rows, in one CTA.
// Consecutive x share DRAM sectors (G[r, r^x] and G[r, r^x^1] are adjacent), and their
// coefficients n(x, z), n(x^1, z) are adjacent too, so a unit reads and writes whole sectors.
// For N >= 13 a unit is one class pair (x, x^1) over all rows, shared by a cluster of
// 2^(N-12) CTAs (see xordiag_cluster_kernel).
// The transform runs in register phases of up to 4 butterfly stages, with the data
// re-distributed between threads through shared memory (XOR-swizzled 16-byte slots).
// One unit per CTA (cluster), in blockIdx order; where it pays, each CTA prefetches into L2
// the rows of the unit one resident wave ahead, so HBM stays busy during the arithmetic.
// Decompositions at N = 13, 14 default to the two-stage tiled kernel (tiled_impl.cuh).
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
#include "tiled.h"

namespace pauli {

cudaError_t xordiag_c128_decompose(int, int, const void*, long long, int, void*, cudaStream_t);
cudaError_t xordiag_c128_compose(int, int, const void*, long long, int, void*, cudaStream_t);
cudaError_t xordiag_c64_decompose(int, int, const void*, long long, int, void*, cudaStream_t);
cudaError_t xordiag_c64_compose(int, int, const void*, long long, int, void*, cudaStream_t);
cudaError_t xordiag_re_decompose_c128(int, const void*, long long, void*, cudaStream_t, bool);
cudaError_t xordiag_re_decompose_c64(int, const void*, long long, void*, cudaStream_t, bool);
cudaError_t xordiag_herm_upper_c128(int, const void*, long long, void*, cudaStream_t);
cudaError_t xordiag_real_decompose(int, const void*, long long, void*, cudaStream_t, bool);
cudaError_t tiled_launch_real_r4(const void*, int, int, void*, cudaStream_t);
cudaError_t xordiag_herm_upper_c64(int, const void*, long long, void*, cudaStream_t);

namespace {

bool is_tiled(int v) { return v == kVariantTiled8 || v == kVariantTiled16 || v == kVariantTwoStage; }
// Consumer shape argument of launch_tiled: 3 / 4 = block-tiled kernel, 0 = warp-independent kernel.
int tiled_rb(int v) { return v == kVariantTiled8 ? 3 : v == kVariantTiled16 ? 4 : 0; }

bool variant_has(int variant, int N, bool compose) {
  if (variant == kVariantUnit13 || variant == kVariantUnit13x8) return N >= 7 && N <= 15;
  if (variant == kVariantUnit12 || variant == kVariantUnit12x8) return N >= 6 && N <= 14;
  if (is_tiled(variant)) return !compose && tiled_supported(N);
  return false;
}

// The tiled kernel numbers its work items with 32-bit integers.
constexpr long long kTiledMaxCount = 1024;

// Chosen variant per (one matrix or a batch, N, dtype, direction): 0 = built-in default. Set
// by the autotuner.
int g_variant[2][2][2][17];

// Built-in choice (measured on GB300): the warp-independent two-stage kernel for decompositions
// at N = 12..14 (N = 14: 2.40 ms complex128 and 2.10 ms complex64, against 2.60 and 3.12 ms for the
// block-tiled kernel; N = 12: 0.186 / 0.143 ms against 0.186 / 0.176 ms single-pass), else single-pass units of 8192 (4096 below N = 7) elements; for batches
// of matrices below N = 12, 4096-element units on two CTAs per SM (64 x N = 10: 0.46 instead of
// 0.50 ms).
int default_variant(int N, bool c64, bool compose, bool batched) {
  (void)c64;
  if (!compose && N >= 12 && N <= 14) return kVariantTwoStage;
  if (batched && N < 12) return kVariantUnit12;
  return N >= 7 ? kVariantUnit13 : kVariantUnit12;
}
// The single-pass choice, for requests the tiled kernel cannot take.
int single_pass_variant(int N) { return N >= 7 ? kVariantUnit13 : kVariantUnit12; }

}  // namespace

bool xordiag_supported(int N) { return N >= 6 && N <= 15; }

bool xordiag_variant_supported(int variant, int N, bool compose) { return variant_has(variant, N, compose); }

int xordiag_get_variant(int N, bool c64, bool compose, bool batched) {
  if (N < 0 || N > 16) return 0;
  const int v = g_variant[batched][c64][compose][N];
  return v ? v : (xordiag_supported(N) ? default_variant(N, c64, compose, batched) : 0);
}

void xordiag_set_variant(int N, bool c64, bool compose, bool batched, int variant) {
  if (N >= 0 && N <= 16) g_variant[batched][c64][compose][N] = variant;
}

cudaError_t launch_xordiag(const void* in, int N, long long count, bool c64, bool compose, int scale_exp, void* out,
                           cudaStream_t s, int variant) {
  if (!variant) {
    variant = xordiag_get_variant(N, c64, compose, count > 1);
    if (is_tiled(variant) &&
        (count > kTiledMaxCount || (reinterpret_cast<uintptr_t>(in) & 15u)))
      variant = single_pass_variant(N);
  }
  if (!variant_has(variant, N, compose)) return cudaErrorNotSupported;
  if (is_tiled(variant)) {
    // the bulk copies need 16-byte aligned sources: other G take the single-pass kernel
    if (count > kTiledMaxCount || (reinterpret_cast<uintptr_t>(in) & 15u))
      return launch_xordiag(in, N, count, c64, compose, scale_exp, out, s, single_pass_variant(N));
    return launch_tiled(in, N, (int)count, c64, out, tiled_rb(variant), s);
  }
  if (c64)
    return compose ? xordiag_c64_compose(variant, N, in, count, scale_exp, out, s)
                   : xordiag_c64_decompose(variant, N, in, count, scale_exp, out, s);
  return compose ? xordiag_c128_compose(variant, N, in, count, scale_exp, out, s)
                 : xordiag_c128_decompose(variant, N, in, count, scale_exp, out, s);
}

// Real parts only: the tiled kernel where the decomposition's chosen shape is tiled (and the
// batch and alignment allow it), else single-pass units of the chosen size with 16 elements
// per thread.
cudaError_t launch_xordiag_re(const void* in, int N, long long count, bool c64, void* out, cudaStream_t s) {
  if (!xordiag_supported(N)) return cudaErrorNotSupported;
  const int v = xordiag_get_variant(N, c64, false, count > 1);
  if (is_tiled(v) && tiled_supported(N) && count <= kTiledMaxCount && !(reinterpret_cast<uintptr_t>(in) & 15u))
    return launch_tiled(in, N, (int)count, c64, out, tiled_rb(v), s, true);
  const bool unit4096 = (v == kVariantUnit12 || v == kVariantUnit12x8) && N <= 14;
  return c64 ? xordiag_re_decompose_c64(N, in, count, out, s, unit4096)
             : xordiag_re_decompose_c128(N, in, count, out, s, unit4096);
}

// Real (float64) input: the tiled kernel where the complex128 decomposition's chosen shape is
// tiled (16 elements per thread), else single-pass units of the chosen size.
cudaError_t launch_xordiag_real(const void* in, int N, long long count, void* out, cudaStream_t s) {
  if (!xordiag_supported(N)) return cudaErrorNotSupported;
  const int v = xordiag_get_variant(N, false, false, count > 1);
  if (is_tiled(v) && tiled_supported(N) && count <= kTiledMaxCount &&
      !(reinterpret_cast<uintptr_t>(in) & 15u))
    return tiled_launch_real_r4(in, N, (int)count, out, s);
  const bool unit4096 = (v == kVariantUnit12 || v == kVariantUnit12x8) && N <= 14;
  return xordiag_real_decompose(N, in, count, out, s, unit4096);
}

cudaError_t launch_xordiag_herm_upper(const void* G, int N, long long count, bool c64, void* out, cudaStream_t s) {
  return c64 ? xordiag_herm_upper_c64(N, G, count, out, s) : xordiag_herm_upper_c128(N, G, count, out, s);
}

}  // namespace pauli

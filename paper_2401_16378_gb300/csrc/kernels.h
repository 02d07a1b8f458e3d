// kernels.h -- internal launch functions of libpauli (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pauli {

// Eq. (13) per coefficient, Gray-code order (plain.cu).
// re: store only Re c_n, into count * 4^N reals; upper (with re): G Hermitian, read from its
// upper triangle.
cudaError_t launch_plain_decompose(const void* G, int N, long long count, bool c64, void* out, cudaStream_t s,
                                   bool re = false, bool upper = false);
// Real (float64) G: count * 4^N reals a_n with c_n = i^(k mod 2) a_n, k the number of Y factors
// of P_n (xordiag_real.cu, tiled_real_r4.cu).
cudaError_t launch_xordiag_real(const void* G, int N, long long count, void* out, cudaStream_t s);
cudaError_t launch_plain_decompose_real(const void* G, int N, long long count, void* out, cudaStream_t s);
// Hermitian G read from its upper triangle, real coefficients, N = 7..12 (xordiag_herm_*.cu).
cudaError_t launch_xordiag_herm_upper(const void* G, int N, long long count, bool c64, void* out, cudaStream_t s);
// The same for N = 12..14 with the two-stage kernel in its upper-triangle mode (count <= 1024,
// G 16-byte aligned; tiled.cu).
cudaError_t twostage_launch_upper(const void* G, int N, int count, bool c64, void* out, cudaStream_t s);
// w, g (nullable): compose g w_n c_n instead of c_n.
cudaError_t launch_plain_compose(const void* c, int N, long long count, bool c64, int scale_exp, void* G,
                                cudaStream_t s, const void* w = nullptr, const void* g = nullptr);
cudaError_t launch_coeffs_at(const void* G, int N, bool c64, const uint64_t* idx, long long k, void* out,
                             cudaStream_t s);

// XOR-diagonal gather + Walsh-Hadamard transform (xordiag.cu). compose = the inverse map
// scaled by 2^scale_exp. Returns cudaErrorNotSupported when N has no XOR-diagonal kernel.
// Variants (launch shapes): 8192-element units on 512-thread CTAs, or 4096-element units on
// 256-thread CTAs (two per SM); 0 selects the tuned or built-in choice.
constexpr int kVariantUnit13 = 1;    // 8192-element units, 512 threads x 16 elements
constexpr int kVariantUnit12 = 2;    // 4096-element units, 256 threads x 16 elements, 2 CTAs/SM
constexpr int kVariantUnit12x8 = 3;  // 4096-element units, 512 threads x 8 elements, 2 CTAs/SM
constexpr int kVariantUnit13x8 = 4;  // 8192-element units, 1024 threads x 8 elements
constexpr int kVariantTiled8 = 5;    // two-stage tiled decomposition (tiled.cu), 512 consumers x 8 elements
constexpr int kVariantTiled16 = 6;   // two-stage tiled decomposition, 256 consumers x 16 elements
constexpr int kVariantTwoStage = 7;  // two-stage decomposition with warp-independent consumers
bool xordiag_supported(int N);
bool xordiag_variant_supported(int variant, int N, bool compose);
// batched: the choice for calls with count > 1 (kept apart from the one-matrix choice).
int xordiag_get_variant(int N, bool c64, bool compose, bool batched);
void xordiag_set_variant(int N, bool c64, bool compose, bool batched, int variant);
cudaError_t launch_xordiag(const void* in, int N, long long count, bool c64, bool compose, int scale_exp, void* out,
                           cudaStream_t s, int variant = 0);
// Decomposition storing only Re c_n, into count * 4^N reals (double / float).
cudaError_t launch_xordiag_re(const void* in, int N, long long count, bool c64, void* out, cudaStream_t s);

// Fused forms (fused.cu). Decomposition that also writes L = sum_k sum_n w_n |c_kn|^2
// to *loss (any N: one fused kernel for N 6..12, else decomposition + norm), and composition of
// g w_n c_n (N <= 12; cudaErrorNotSupported above).
cudaError_t launch_decompose_norm(const void* G, int N, long long count, bool c64, void* out, const void* w,
                                  void* loss, int method, cudaStream_t s);
cudaError_t launch_compose_weighted(const void* c, int N, long long count, bool c64, const void* w, const void* g,
                                    int scale_exp, void* G, cudaStream_t s);
// Composition of a batch of coefficient vectors of uneven N (1 <= N <= compose_batched_max_n()),
// host arrays of device pointers; one launch per 1024 matrices (compose_batched.cu).
int compose_batched_max_n();
cudaError_t launch_compose_batched(const void* const* c_list, const int* N_list, int batch, bool c64,
                                   void* const* G_list, int scale_exp, cudaStream_t s);
// x-class shards (xhi.cu): the in-place combine of 2^k stacked (N - k)-qubit decompositions
// into the coefficients with top XY-mask bits x_hi, and the block-XOR copy of G that feeds it.
cudaError_t launch_xhi_combine(void* out, int N, int k, uint32_t x_hi, bool c64, cudaStream_t s);
// The shard in one two-stage launch from its layout (N 12..14, N - k >= 6, L 16-byte aligned):
// cudaErrorNotSupported otherwise (twostage_*.cu).
cudaError_t twostage_launch_xhi(const void* L, int N, int k, uint32_t x_hi, bool c64, void* out, cudaStream_t s);
cudaError_t xhi_layout(const void* G, int N, int k, uint32_t x_hi, size_t elem, void* L, cudaStream_t s);
// Adds n partial losses (fixed order) into *loss (norm.cu).
cudaError_t launch_norm_final(const double* partial, long long n, bool c64, void* loss, cudaStream_t s);

// Weighted coefficient norm L = sum_k sum_n w_n |c_{k,n}|^2 (two launches, deterministic) and
// its gradient grad_c = 2 g w_n c (one launch; grad_c may be c) (norm.cu). w and the outputs are
// double for complex128, float for complex64; g is a device scalar or nullptr (g = 1).
cudaError_t launch_weighted_norm(const void* c, int N, long long count, bool c64, const void* w, void* loss,
                                 cudaStream_t s);
cudaError_t launch_weighted_norm_grad(const void* c, int N, long long count, bool c64, const void* w, const void* g,
                                      void* grad_c, cudaStream_t s);

}  // namespace pauli

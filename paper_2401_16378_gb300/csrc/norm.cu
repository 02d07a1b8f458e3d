// norm.cu -- the weighted coefficient norm of a batch of coefficient vectors and its
// gradient with respect to the coefficients:
//   L = sum_k sum_n w_n |c_{k,n}|^2,      dL/dc_{k,n} = 2 g w_n c_{k,n}
// (the gradient in PyTorch's convention for complex inputs, times the incoming gradient g of
// L). With c = decompose(G) this is the real loss whose gradient the adjoint of the linear
// map of Eq. (4) carries back to G; for w = 1 it is 2^-N ||G||_F^2, because the Pauli tensors
// are orthogonal, Tr(P_m P_n) = 2^N [m = n] (Sec. 2).
//
// Both are single passes over c, bound by HBM (16 bytes read per complex128 element; the
// gradient also writes 16). FP64 issues at about 2 operations per clock per SM on this GPU,
// so the complex128 kernels spend at most 2 FP64 operations per element: when the batch has
// several vectors a thread owns a coefficient index n, runs over the batch accumulating
// |c_{k,n}|^2 (or scaling by its one factor 2 g w_n), and applies w_n once.
//
// The sum is deterministic: a fixed grid of kBlocks x kThreads threads, a fixed order within
// each thread, a fixed tree within each block, and a second one-block kernel that adds the
// kBlocks partials in a fixed tree.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "workspace.h"

namespace pauli {
namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 1024;
constexpr int kLogP = 18;  // log2(kBlocks * kThreads)
constexpr unsigned long long kP = 1ull << kLogP;
static_assert((1ull << kLogP) == (unsigned long long)kBlocks * kThreads, "grid size");
// Batches of at least this many vectors take the per-n form (w applied once per n).
constexpr long long kColumnMinCount = 4;

// Sum of v over the block (fixed tree); the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double part[kThreads / 32];
#pragma unroll
  for (int m = 16; m; m >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
  if ((threadIdx.x & 31u) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < kThreads / 32; ++i) s += part[i];
  }
  return s;
}

// Compensated FP32 accumulator (Knuth's TwoSum per addition): the running sum s and the
// accumulated rounding errors e of its additions.
struct F32Sum {
  float s = 0.f, e = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float bp = t - s;
    e += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)e; }
};

// ---- complex128, per-n form: thread owns n = tid + j P (4^N >= P) or one n and every
// (P / 4^N)-th vector of the batch (4^N < P).
__global__ void __launch_bounds__(kThreads) norm_c128_columns(const double2* __restrict__ c,
                                                              const double* __restrict__ w, int N,
                                                              long long count, double* __restrict__ partial) {
  const unsigned long long M = 1ull << (2 * N);
  const unsigned long long tid = (unsigned long long)blockIdx.x * kThreads + threadIdx.x;
  unsigned long long n0 = tid, nstep = kP;
  long long k0 = 0, kstep = 1;
  if (M < kP) {
    n0 = tid & (M - 1);
    nstep = M;
    k0 = (long long)(tid >> (2 * N));
    kstep = (long long)(kP >> (2 * N));
  }
  double total = 0.0;
  for (unsigned long long n = n0; n < M; n += nstep) {
    const double2* col = c + n;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    long long k = k0;
    for (; k + 3 * kstep < count; k += 4 * kstep) {
      const double2 v0 = col[(unsigned long long)k * M];
      const double2 v1 = col[(unsigned long long)(k + kstep) * M];
      const double2 v2 = col[(unsigned long long)(k + 2 * kstep) * M];
      const double2 v3 = col[(unsigned long long)(k + 3 * kstep) * M];
      a0 = fma(v0.y, v0.y, fma(v0.x, v0.x, a0));
      a1 = fma(v1.y, v1.y, fma(v1.x, v1.x, a1));
      a2 = fma(v2.y, v2.y, fma(v2.x, v2.x, a2));
      a3 = fma(v3.y, v3.y, fma(v3.x, v3.x, a3));
    }
    for (; k < count; k += kstep) {
      const double2 v = col[(unsigned long long)k * M];
      a0 = fma(v.y, v.y, fma(v.x, v.x, a0));
    }
    total = fma(w[n], (a0 + a1) + (a2 + a3), total);
  }
  const double s = block_sum(total);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// ---- flat form: element i = tid + j P of the whole batch, n = i mod 4^N.
template <bool C64>
__global__ void __launch_bounds__(kThreads) norm_flat(const void* __restrict__ cv, const void* __restrict__ wv,
                                                      int N, unsigned long long total_elems,
                                                      double* __restrict__ partial) {
  const unsigned long long mask = (1ull << (2 * N)) - 1ull;
  const unsigned long long tid = (unsigned long long)blockIdx.x * kThreads + threadIdx.x;
  double t = 0.0;
  if constexpr (C64) {
    const float2* c = static_cast<const float2*>(cv);
    const float* w = static_cast<const float*>(wv);
    F32Sum acc;
    unsigned long long i = tid;
    for (; i + 3 * kP < total_elems; i += 4 * kP) {
      float2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = c[i + u * kP];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc.add(w[(i + u * kP) & mask] * fmaf(v[u].y, v[u].y, v[u].x * v[u].x));
    }
    for (; i < total_elems; i += kP) {
      const float2 v = c[i];
      acc.add(w[i & mask] * fmaf(v.y, v.y, v.x * v.x));
    }
    t = acc.value();
  } else {
    const double2* c = static_cast<const double2*>(cv);
    const double* w = static_cast<const double*>(wv);
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    unsigned long long i = tid;
    for (; i + 3 * kP < total_elems; i += 4 * kP) {
      double2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = c[i + u * kP];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = fma(w[(i + u * kP) & mask], fma(v[u].y, v[u].y, v[u].x * v[u].x), a[u]);
    }
    for (; i < total_elems; i += kP) {
      const double2 v = c[i];
      a[0] = fma(w[i & mask], fma(v.y, v.y, v.x * v.x), a[0]);
    }
    t = (a[0] + a[1]) + (a[2] + a[3]);
  }
  const double s = block_sum(t);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Adds n partials (thread t: partials t, t + 1024, ... in order, then a fixed tree) and writes
// L in the output's real type.
template <bool C64>
__global__ void __launch_bounds__(1024) norm_final(const double* __restrict__ partial, long long n,
                                                   void* __restrict__ loss) {
  __shared__ double part[32];
  double v = 0.0;
  for (long long i = threadIdx.x; i < n; i += 1024) v += partial[i];
#pragma unroll
  for (int m = 16; m; m >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
  if ((threadIdx.x & 31u) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = part[threadIdx.x];
#pragma unroll
    for (int m = 16; m; m >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, m);
    if (threadIdx.x == 0) {
      if constexpr (C64)
        *static_cast<float*>(loss) = (float)v;
      else
        *static_cast<double*>(loss) = v;
    }
  }
}

// ---- gradient, complex128 per-n form: grad[k, n] = f_n c[k, n], f_n = 2 g w_n.
__global__ void __launch_bounds__(kThreads) grad_c128_columns(const double2* c, const double* __restrict__ w,
                                                              const double* __restrict__ g, int N, long long count,
                                                              double2* out) {
  const unsigned long long M = 1ull << (2 * N);
  const unsigned long long tid = (unsigned long long)blockIdx.x * kThreads + threadIdx.x;
  unsigned long long n0 = tid, nstep = kP;
  long long k0 = 0, kstep = 1;
  if (M < kP) {
    n0 = tid & (M - 1);
    nstep = M;
    k0 = (long long)(tid >> (2 * N));
    kstep = (long long)(kP >> (2 * N));
  }
  const double two_g = 2.0 * (g ? *g : 1.0);
  for (unsigned long long n = n0; n < M; n += nstep) {
    const double f = two_g * w[n];
    long long k = k0;
    for (; k + 3 * kstep < count; k += 4 * kstep) {
      double2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = c[(unsigned long long)(k + u * kstep) * M + n];
#pragma unroll
      for (int u = 0; u < 4; ++u) out[(unsigned long long)(k + u * kstep) * M + n] = make_double2(f * v[u].x, f * v[u].y);
    }
    for (; k < count; k += kstep) {
      const double2 v = c[(unsigned long long)k * M + n];
      out[(unsigned long long)k * M + n] = make_double2(f * v.x, f * v.y);
    }
  }
}

// ---- gradient, flat form.
template <bool C64>
__global__ void __launch_bounds__(kThreads) grad_flat(const void* cv, const void* __restrict__ wv,
                                                      const void* __restrict__ gv, int N,
                                                      unsigned long long total_elems, void* outv) {
  const unsigned long long mask = (1ull << (2 * N)) - 1ull;
  const unsigned long long tid = (unsigned long long)blockIdx.x * kThreads + threadIdx.x;
  if constexpr (C64) {
    const float2* c = static_cast<const float2*>(cv);
    const float* w = static_cast<const float*>(wv);
    float2* out = static_cast<float2*>(outv);
    const float two_g = 2.0f * (gv ? *static_cast<const float*>(gv) : 1.0f);
    unsigned long long i = tid;
    for (; i + 3 * kP < total_elems; i += 4 * kP) {
      float2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = c[i + u * kP];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float f = two_g * w[(i + u * kP) & mask];
        out[i + u * kP] = make_float2(f * v[u].x, f * v[u].y);
      }
    }
    for (; i < total_elems; i += kP) {
      const float2 v = c[i];
      const float f = two_g * w[i & mask];
      out[i] = make_float2(f * v.x, f * v.y);
    }
  } else {
    const double2* c = static_cast<const double2*>(cv);
    const double* w = static_cast<const double*>(wv);
    double2* out = static_cast<double2*>(outv);
    const double two_g = 2.0 * (gv ? *static_cast<const double*>(gv) : 1.0);
    unsigned long long i = tid;
    for (; i + 3 * kP < total_elems; i += 4 * kP) {
      double2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = c[i + u * kP];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double f = two_g * w[(i + u * kP) & mask];
        out[i + u * kP] = make_double2(f * v[u].x, f * v[u].y);
      }
    }
    for (; i < total_elems; i += kP) {
      const double2 v = c[i];
      const double f = two_g * w[i & mask];
      out[i] = make_double2(f * v.x, f * v.y);
    }
  }
}

}  // namespace

cudaError_t launch_weighted_norm(const void* c, int N, long long count, bool c64, const void* w, void* loss,
                                 cudaStream_t st) {
  void* ws = nullptr;
  cudaError_t e = stream_workspace(kWorkspaceNorm, st, kBlocks * sizeof(double), kNormWorkspaceReserve, 0, &ws);
  if (e != cudaSuccess) return e;
  double* partial = static_cast<double*>(ws);
  const unsigned long long total = (unsigned long long)count << (2 * N);
  if (c64)
    norm_flat<true><<<kBlocks, kThreads, 0, st>>>(c, w, N, total, partial);
  else if (count >= kColumnMinCount)
    norm_c128_columns<<<kBlocks, kThreads, 0, st>>>(static_cast<const double2*>(c), static_cast<const double*>(w),
                                                     N, count, partial);
  else
    norm_flat<false><<<kBlocks, kThreads, 0, st>>>(c, w, N, total, partial);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_norm_final(partial, kBlocks, c64, loss, st);
}

cudaError_t launch_norm_final(const double* partial, long long n, bool c64, void* loss, cudaStream_t st) {
  if (c64)
    norm_final<true><<<1, 1024, 0, st>>>(partial, n, loss);
  else
    norm_final<false><<<1, 1024, 0, st>>>(partial, n, loss);
  return cudaGetLastError();
}

cudaError_t launch_weighted_norm_grad(const void* c, int N, long long count, bool c64, const void* w, const void* g,
                                      void* grad_c, cudaStream_t st) {
  const unsigned long long total = (unsigned long long)count << (2 * N);
  if (c64)
    grad_flat<true><<<kBlocks, kThreads, 0, st>>>(c, w, g, N, total, grad_c);
  else if (count >= kColumnMinCount)
    grad_c128_columns<<<kBlocks, kThreads, 0, st>>>(static_cast<const double2*>(c), static_cast<const double*>(w),
                                                     static_cast<const double*>(g), N, count,
                                                     static_cast<double2*>(grad_c));
  else
    grad_flat<false><<<kBlocks, kThreads, 0, st>>>(c, w, g, N, total, grad_c);
  return cudaGetLastError();
}

}  // namespace pauli

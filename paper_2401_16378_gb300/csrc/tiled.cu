// tiled.cu -- host side of the two-stage tiled decomposition: its scratch workspace per
// (device, stream), the tensor map, dispatch to the per-shape instantiations, and the status word.
// The kernel and the algorithm are in tiled_impl.cuh.
#include <atomic>
#include <cstddef>
#include <mutex>

#include <cuda.h>

#include "kernels.h"
#include "tiled.h"
#include "workspace.h"

namespace pauli {

cudaError_t tiled_launch_c128_r3(const void*, int, int, void*, cudaStream_t);
cudaError_t tiled_launch_c128_r4(const void*, int, int, void*, cudaStream_t);
cudaError_t tiled_launch_c64_r3(const void*, int, int, void*, cudaStream_t);
cudaError_t tiled_launch_c64_r4(const void*, int, int, void*, cudaStream_t);
cudaError_t tiled_launch_re_c128_r3(const void*, int, int, void*, cudaStream_t);
cudaError_t tiled_launch_re_c128_r4(const void*, int, int, void*, cudaStream_t);
cudaError_t tiled_launch_re_c64_r3(const void*, int, int, void*, cudaStream_t);
cudaError_t tiled_launch_re_c64_r4(const void*, int, int, void*, cudaStream_t);
cudaError_t twostage_launch_c128(const void*, int, int, void*, cudaStream_t);
cudaError_t twostage_launch_c64(const void*, int, int, void*, cudaStream_t);
cudaError_t twostage_launch_re_c128(const void*, int, int, void*, cudaStream_t);
cudaError_t twostage_launch_re_c64(const void*, int, int, void*, cudaStream_t);
size_t twostage_workspace_bytes_c128(int N);
cudaError_t twostage_launch_upper_c128(const void*, int, int, void*, cudaStream_t);
cudaError_t twostage_launch_upper_c64(const void*, int, int, void*, cudaStream_t);

cudaError_t twostage_launch_upper(const void* G, int N, int count, bool c64, void* out, cudaStream_t s) {
  if (!tiled_supported(N) || count < 1 || count > 1024) return cudaErrorNotSupported;
  return c64 ? twostage_launch_upper_c64(G, N, count, out, s) : twostage_launch_upper_c128(G, N, count, out, s);
}

// The first buffer of a stream is sized for every N, so that it is never replaced.
cudaError_t tiled_workspace(cudaStream_t st, size_t bytes, void** out) {
  return stream_workspace(kWorkspaceTiled, st, bytes, tiled_workspace_max_bytes(), kTiledCtrlBytes, out);
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no link to libcuda).
EncodeTiled encode_tiled() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

}  // namespace

cudaError_t tiled_tensor_map(CUtensorMap* map, const void* G, int N, int count, int elem) {
  EncodeTiled fn = encode_tiled();
  if (!fn) return cudaErrorNotSupported;
  // `count` stacked D x D matrices as one (count D) x (D elem / 8) array of 8-byte words;
  // a box is 64 rows of 64 elements
  const cuuint64_t D = 1ull << N;
  const cuuint64_t dims[2] = {D * (cuuint64_t)elem / 8, D * (cuuint64_t)count};
  const cuuint64_t strides[1] = {D * (cuuint64_t)elem};
  const cuuint32_t box[2] = {64u * (cuuint32_t)elem / 8, 64u};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(G), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tiled_tensor_map_rows(CUtensorMap* map, const void* G, int wlog, long long rows, int elem) {
  EncodeTiled fn = encode_tiled();
  if (!fn) return cudaErrorNotSupported;
  // `rows` rows of 2^wlog elements as a rows x (2^wlog elem / 8) array of 8-byte words; a box is
  // 64 rows of 64 elements
  const cuuint64_t W = 1ull << wlog;
  const cuuint64_t dims[2] = {W * (cuuint64_t)elem / 8, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {W * (cuuint64_t)elem};
  const cuuint32_t box[2] = {64u * (cuuint32_t)elem / 8, 64u};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(G), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t scratch_tensor_map(CUtensorMap* map, void* base, long long rows, int row_words, int box_words,
                               int box_rows) {
  EncodeTiled fn = encode_tiled();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)row_words, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)row_words * 8u};
  const cuuint32_t box[2] = {(cuuint32_t)box_words, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 4D map of stage-2 chunks: (words of one warp's transforms, tile R, warp slice, chunk) over the
// dense [chunk][R][slice][words] scratch; a box of one chunk lands as [slice][R][words].
cudaError_t scratch_tensor_map4(CUtensorMap* map, void* base, int chunks, int nr, int slice_words) {
  auto fn = encode_tiled();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t row = (cuuint64_t)slice_words * 8u * 8u;  // bytes of one R row: 8 slices
  const cuuint64_t dims[4] = {(cuuint64_t)slice_words, (cuuint64_t)nr, 8u, (cuuint64_t)chunks};
  const cuuint64_t strides[3] = {row, (cuuint64_t)slice_words * 8u, row * (cuuint64_t)nr};
  const cuuint32_t box[4] = {(cuuint32_t)slice_words, (cuuint32_t)nr, 8u, 1u};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace {
std::atomic<bool> g_stall_next{false};
}  // namespace

void tiled_debug_stall_next() { g_stall_next.store(true); }
bool tiled_take_stall() { return g_stall_next.exchange(false); }

bool tiled_supported(int N) { return N >= 12 && N <= 14; }

cudaError_t launch_tiled(const void* G, int N, int count, bool c64, void* out, int rb, cudaStream_t st, bool re) {
  if (!tiled_supported(N)) return cudaErrorNotSupported;
  if (rb == 0) {  // the warp-independent two-stage kernel
    using Fn = cudaError_t (*)(const void*, int, int, void*, cudaStream_t);
    static const Fn ts_table[2][2] = {{twostage_launch_c128, twostage_launch_c64},
                                      {twostage_launch_re_c128, twostage_launch_re_c64}};
    return ts_table[re][c64](G, N, count, out, st);
  }
  using Fn = cudaError_t (*)(const void*, int, int, void*, cudaStream_t);
  static const Fn table[2][2][2] = {  // [re][c64][rb == 4]
      {{tiled_launch_c128_r3, tiled_launch_c128_r4}, {tiled_launch_c64_r3, tiled_launch_c64_r4}},
      {{tiled_launch_re_c128_r3, tiled_launch_re_c128_r4}, {tiled_launch_re_c64_r3, tiled_launch_re_c64_r4}}};
  if (rb != 3 && rb != 4) return cudaErrorNotSupported;
  return table[re][c64][rb == 4](G, N, count, out, st);
}

cudaError_t tiled_stream_status(cudaStream_t st, int* status) {
  *status = 0;
  void* p = stream_workspace_find(kWorkspaceTiled, st);
  if (!p) return cudaSuccess;
  cudaError_t e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  int* sp = reinterpret_cast<int*>(reinterpret_cast<char*>(p) + offsetof(TiledCtrl, status));
  if ((e = cudaMemcpyAsync(status, sp, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(sp, 0, sizeof(int), st)) != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

}  // namespace pauli

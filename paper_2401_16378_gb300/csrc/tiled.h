// tiled.h -- the two-stage XOR-diagonal decomposition for large N (tiled.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace pauli {

constexpr int kTiledSlots = 3;           // scratch ring slots
constexpr size_t kTiledCtrlBytes = 256;  // control block, padded so the slots start 256-byte aligned

// Device control block at the start of the workspace; cleared before every launch except
// `status`, which keeps the first error until pauli_stream_status reads and clears it.
struct TiledCtrl {
  int counter;                 // next work item
  int s1_done[kTiledSlots];    // stage-1 tiles completed per slot (all generations)
  int s2_done[kTiledSlots];    // stage-2 items that have read their slot (all generations)
  int pad;
  int status;                  // PAULI_OK or PAULI_ERR_TIMEOUT
};

bool tiled_supported(int N);
// Unit size (log2 elements) of the tiled launch: 13 (512 threads, one CTA per SM) or 12 (256
// threads, two CTAs per SM).
cudaError_t launch_tiled(const void* G, int N, int count, bool c64, void* out, int unit_bits, cudaStream_t st);
// Status word of the workspace used on `st` (synchronises st); 0 when none exists.
cudaError_t tiled_stream_status(cudaStream_t st, int* status);

}  // namespace pauli

// tiled.h -- the two-stage XOR-diagonal decomposition for large N (tiled.cu, tiled_impl.cuh).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

namespace pauli {

constexpr int kTiledSlots = 16;  // most scratch ring slots (the ring depth is chosen per N)

// Device control block at the start of the workspace. Everything from `counter` on is
// cleared before every launch; `status` keeps the first error until pauli_stream_status reads
// and clears it.
struct TiledCtrl {
  int status;  // PAULI_OK or PAULI_ERR_TIMEOUT
  int pad0[3];
  int counter;                  // next work item
  int s1_done[kTiledSlots];     // stage-1 tiles completed per slot (all generations)
  int s2_done[kTiledSlots];     // stage-2 items that have copied their slot's data (all generations)
  int stall;                    // test hook: the producer's first wait waits on a count nothing raises
  int pad1[6];
  uint32_t emax[kTiledSlots][64];  // per class of the slot's block: (generation + 1) << 11 | exponent
};
constexpr size_t kTiledCtrlBytes = 8192;  // control block, padded; the slots follow
static_assert(sizeof(TiledCtrl) <= kTiledCtrlBytes, "control block fits its padding");

bool tiled_supported(int N);
// Scratch bytes a tiled launch at N needs (0 when N has no tiled kernel), and the most over N.
size_t tiled_workspace_bytes(int N);
size_t tiled_workspace_max_bytes();
// rb = log2 of the elements per consumer thread: 3 (512 consumer threads) or 4 (256).
// re: store only the real parts, into an array of reals (Hermitian decomposition).
cudaError_t launch_tiled(const void* G, int N, int count, bool c64, void* out, int rb, cudaStream_t st,
                         bool re = false);
// Status word of the workspace used on `st` (synchronises st); 0 when none exists.
cudaError_t tiled_stream_status(cudaStream_t st, int* status);
// Test hook: the next tiled launch (any stream) stalls its producers on a wait that nothing
// satisfies; the bounded wait gives up and records PAULI_ERR_TIMEOUT.
void tiled_debug_stall_next();
bool tiled_take_stall();

}  // namespace pauli

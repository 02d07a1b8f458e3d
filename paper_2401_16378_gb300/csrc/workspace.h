// workspace.h -- device scratch buffers kept per (device, stream, kind) for the life of the
// process, and caller-provided scratch for one call (workspace.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace pauli {

enum WorkspaceKind { kWorkspaceTiled = 0, kWorkspaceNorm = 1 };

// First size of a per-stream buffer of the weighted norm: 8-byte partials of 4096-element units,
// enough for batches of up to 2^29 elements before a larger request replaces it.
constexpr size_t kNormWorkspaceReserve = (size_t)1 << 20;

// A buffer of at least `bytes` for (current device, st, kind). The first buffer of a
// (device, stream, kind) is allocated with max(bytes, reserve) bytes so that later calls with
// up to `reserve` bytes reuse it; a request beyond the buffer's size replaces it (cudaFree waits
// for the device, so no launch still uses the old one). A new buffer has its first
// `clear_bytes` zeroed on st. While a caller workspace is active on this thread (below), a
// request of that kind is served from it and nothing is allocated.
cudaError_t stream_workspace(int kind, cudaStream_t st, size_t bytes, size_t reserve, size_t clear_bytes, void** out);
// The existing buffer for (current device, st, kind), or nullptr.
void* stream_workspace_find(int kind, cudaStream_t st);
// Synchronises st and frees every buffer of (current device, st).
cudaError_t stream_workspace_release(cudaStream_t st);

// Caller-provided scratch of one kind for the calls made on this thread while the object lives
// (the entry points that take a workspace argument). A request larger than `bytes` fails with
// cudaErrorInvalidValue instead of allocating.
class CallerWorkspace {
 public:
  CallerWorkspace(int kind, void* ptr, size_t bytes);
  ~CallerWorkspace();
  CallerWorkspace(const CallerWorkspace&) = delete;
  CallerWorkspace& operator=(const CallerWorkspace&) = delete;

 private:
  int kind_;
  void* prev_ptr_;
  size_t prev_bytes_;
};

}  // namespace pauli

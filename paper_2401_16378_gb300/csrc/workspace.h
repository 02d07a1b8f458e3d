// workspace.h -- device scratch buffers kept per (device, stream, kind) for the life of the
// process (workspace.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace pauli {

enum WorkspaceKind { kWorkspaceTiled = 0, kWorkspaceNorm = 1 };

// A buffer of at least `bytes` for (current device, st, kind). A new or grown buffer has its
// first `clear_bytes` zeroed on st. Growing frees the old buffer (cudaFree waits for the
// device), so no launch still uses it.
cudaError_t stream_workspace(int kind, cudaStream_t st, size_t bytes, size_t clear_bytes, void** out);
// The existing buffer for (current device, st, kind), or nullptr.
void* stream_workspace_find(int kind, cudaStream_t st);

}  // namespace pauli

// workspace.cu -- device scratch buffers per (device, stream, kind), grown on demand.
#include <mutex>
#include <vector>

#include "workspace.h"

namespace pauli {
namespace {

struct Workspace {
  int dev;
  cudaStream_t stream;
  int kind;
  void* ptr;
  size_t bytes;
};
std::mutex g_mutex;
std::vector<Workspace> g_ws;

}  // namespace

cudaError_t stream_workspace(int kind, cudaStream_t st, size_t bytes, size_t clear_bytes, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mutex);
  Workspace* w = nullptr;
  for (Workspace& x : g_ws)
    if (x.dev == dev && x.stream == st && x.kind == kind) w = &x;
  if (w && w->bytes >= bytes) {
    *out = w->ptr;
    return cudaSuccess;
  }
  if (w) {
    e = cudaFree(w->ptr);
    if (e != cudaSuccess) return e;
    w->ptr = nullptr;
    w->bytes = 0;
  }
  void* p = nullptr;
  e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return e;
  if (clear_bytes) {
    e = cudaMemsetAsync(p, 0, clear_bytes < bytes ? clear_bytes : bytes, st);
    if (e != cudaSuccess) {
      cudaFree(p);
      return e;
    }
  }
  if (w) {
    w->ptr = p;
    w->bytes = bytes;
  } else {
    g_ws.push_back(Workspace{dev, st, kind, p, bytes});
  }
  *out = p;
  return cudaSuccess;
}

void* stream_workspace_find(int kind, cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(g_mutex);
  for (const Workspace& x : g_ws)
    if (x.dev == dev && x.stream == st && x.kind == kind) return x.ptr;
  return nullptr;
}

}  // namespace pauli

// workspace.cu -- device scratch buffers per (device, stream, kind), and caller-provided scratch.
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

constexpr int kKinds = 2;
thread_local void* t_caller_ptr[kKinds] = {};
thread_local size_t t_caller_bytes[kKinds] = {};

}  // namespace

CallerWorkspace::CallerWorkspace(int kind, void* ptr, size_t bytes)
    : kind_(kind), prev_ptr_(t_caller_ptr[kind]), prev_bytes_(t_caller_bytes[kind]) {
  t_caller_ptr[kind] = ptr;
  t_caller_bytes[kind] = bytes;
}

CallerWorkspace::~CallerWorkspace() {
  t_caller_ptr[kind_] = prev_ptr_;
  t_caller_bytes[kind_] = prev_bytes_;
}

cudaError_t stream_workspace(int kind, cudaStream_t st, size_t bytes, size_t reserve, size_t clear_bytes, void** out) {
  if (kind >= 0 && kind < kKinds && t_caller_ptr[kind]) {
    if (bytes > t_caller_bytes[kind]) return cudaErrorInvalidValue;
    *out = t_caller_ptr[kind];
    return cudaSuccess;
  }
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
  const size_t size = bytes > reserve ? bytes : reserve;
  void* p = nullptr;
  e = cudaMalloc(&p, size);
  if (e != cudaSuccess) return e;
  if (clear_bytes) {
    e = cudaMemsetAsync(p, 0, clear_bytes < size ? clear_bytes : size, st);
    if (e != cudaSuccess) {
      cudaFree(p);
      return e;
    }
  }
  if (w) {
    w->ptr = p;
    w->bytes = size;
  } else {
    g_ws.push_back(Workspace{dev, st, kind, p, size});
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

cudaError_t stream_workspace_release(cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mutex);
  for (size_t i = 0; i < g_ws.size();) {
    if (g_ws[i].dev == dev && g_ws[i].stream == st) {
      if ((e = cudaFree(g_ws[i].ptr)) != cudaSuccess) return e;
      g_ws[i] = g_ws.back();
      g_ws.pop_back();
    } else {
      ++i;
    }
  }
  return cudaSuccess;
}

}  // namespace pauli

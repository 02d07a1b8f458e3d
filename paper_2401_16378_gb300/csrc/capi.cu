// capi.cu -- the C ABI of libpauli (include/pauli.h): validation, dispatch, errors, plans.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <algorithm>

#include "kernels.h"
#include "pauli.h"
#include "plan_internal.h"
#include "tiled.h"
#include "workspace.h"

namespace pauli {
int static_batch_max();
int static_batch_launch(const void* const* G_list, const int* N_list, int batch, bool c64, void* const* out_list,
                        cudaStream_t s, const char** what, cudaError_t* cuda_err);
}  // namespace pauli

namespace {

thread_local std::string g_err;
std::atomic<int> g_fail_next{0};

int fail(int status, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return status;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(PAULI_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// Host-side injected launch failure (test hook).
bool take_injected_failure() {
  int n = g_fail_next.load();
  while (n > 0) {
    if (g_fail_next.compare_exchange_weak(n, n - 1)) return true;
  }
  return false;
}

size_t elem_bytes(int dtype) { return dtype == PAULI_C64 ? 8u : 16u; }

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
  return pa < pb + nb && pb < pa + na;
}

int check_dtype(int dtype) {
  if (dtype != PAULI_C64 && dtype != PAULI_C128) return fail(PAULI_ERR_DTYPE, "dtype %d is not PAULI_C64 or PAULI_C128", dtype);
  return PAULI_OK;
}

int check_n(int N) {
  if (N < 1 || N > PAULI_MAX_QUBITS) return fail(PAULI_ERR_ARG, "N = %d outside [1, %d]", N, PAULI_MAX_QUBITS);
  return PAULI_OK;
}

int check_aligned(const void* p, size_t a, const char* name) {
  if ((uintptr_t)p % a) return fail(PAULI_ERR_ALIGN, "%s is not %zu-byte aligned", name, a);
  return PAULI_OK;
}

// Validates a (matrix batch -> coefficient batch) pair; both hold count * 4^N elements.
int check_pair(const void* in, const char* in_name, int N, long long count, int dtype, const void* out,
               const char* out_name) {
  int st;
  if ((st = check_dtype(dtype))) return st;
  if ((st = check_n(N))) return st;
  if (count < 1) return fail(PAULI_ERR_ARG, "count = %lld must be >= 1", count);
  if (!in) return fail(PAULI_ERR_NULL, "%s is NULL", in_name);
  if (!out) return fail(PAULI_ERR_NULL, "%s is NULL", out_name);
  const size_t es = elem_bytes(dtype);
  if ((st = check_aligned(in, es, in_name))) return st;
  if ((st = check_aligned(out, es, out_name))) return st;
  const unsigned long long per = 1ull << (2 * N);
  if ((unsigned long long)count > (~0ull / es) / per) return fail(PAULI_ERR_ARG, "count * 4^N overflows");
  const size_t bytes = (size_t)(per * (unsigned long long)count) * es;
  if (overlaps(in, bytes, out, bytes)) return fail(PAULI_ERR_ALIAS, "%s and %s overlap", in_name, out_name);
  return PAULI_OK;
}

// Validates a (matrix batch -> real coefficient batch) pair: count * 4^N complex inputs and as
// many reals out.
int check_real_out(const void* G, int N, long long count, int dtype, const void* out_re) {
  int st;
  if ((st = check_dtype(dtype))) return st;
  if ((st = check_n(N))) return st;
  if (count < 1) return fail(PAULI_ERR_ARG, "count = %lld must be >= 1", count);
  if (!G) return fail(PAULI_ERR_NULL, "G is NULL");
  if (!out_re) return fail(PAULI_ERR_NULL, "out_re is NULL");
  const size_t es = elem_bytes(dtype);
  if ((st = check_aligned(G, es, "G"))) return st;
  if ((st = check_aligned(out_re, es / 2, "out_re"))) return st;
  const unsigned long long per = 1ull << (2 * N);
  if ((unsigned long long)count > (~0ull / es) / per) return fail(PAULI_ERR_ARG, "count * 4^N overflows");
  const size_t in_bytes = (size_t)(per * (unsigned long long)count) * es;
  if (overlaps(G, in_bytes, out_re, in_bytes / 2)) return fail(PAULI_ERR_ALIAS, "G and out_re overlap");
  return PAULI_OK;
}

int resolve_method(int method, int N, int* out) {
  if (method == PAULI_AUTO) {
    *out = pauli::xordiag_supported(N) ? PAULI_XORDIAG : PAULI_PLAIN;
    return PAULI_OK;
  }
  if (method == PAULI_PLAIN) {
    *out = PAULI_PLAIN;
    return PAULI_OK;
  }
  if (method == PAULI_XORDIAG) {
    if (!pauli::xordiag_supported(N))
      return fail(PAULI_ERR_UNSUPPORTED, "PAULI_XORDIAG is not built for N = %d", N);
    *out = PAULI_XORDIAG;
    return PAULI_OK;
  }
  return fail(PAULI_ERR_ARG, "method %d is not a pauli_method", method);
}

// Library streams of pauli_decompose_host_stream, one set per device, kept for the process:
// copy in, compute, copy out, and the events that order them. Calls on a device take the mutex
// while they enqueue.
struct HostPipe {
  std::mutex mutex;
  cudaStream_t in = nullptr, comp = nullptr, out = nullptr;
  cudaEvent_t start = nullptr, end = nullptr, in_done[2] = {}, comp_done[2] = {}, out_done[2] = {};
};
std::mutex g_pipes_mutex;
std::vector<std::pair<int, HostPipe*>> g_pipes;

cudaError_t host_pipe(HostPipe** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_pipes_mutex);
  for (auto& p : g_pipes)
    if (p.first == dev) {
      *out = p.second;
      return cudaSuccess;
    }
  HostPipe* hp = new (std::nothrow) HostPipe;
  if (!hp) return cudaErrorMemoryAllocation;
  cudaStream_t* streams[] = {&hp->in, &hp->comp, &hp->out};
  cudaEvent_t* events[] = {&hp->start, &hp->end, &hp->in_done[0], &hp->in_done[1], &hp->comp_done[0],
                           &hp->comp_done[1], &hp->out_done[0], &hp->out_done[1]};
  for (cudaStream_t* s : streams)
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
  for (cudaEvent_t* ev : events)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {  // release what was created
    for (cudaEvent_t* ev : events)
      if (*ev) cudaEventDestroy(*ev);
    for (cudaStream_t* s : streams)
      if (*s) cudaStreamDestroy(*s);
    delete hp;
    return e;
  }
  g_pipes.emplace_back(dev, hp);
  *out = hp;
  return cudaSuccess;
}

// Scratch bytes that pauli_decompose takes for these arguments (the tiled kernel's ring), or 0.
int decompose_workspace_bytes(int N, long long count, int dtype, int method, size_t* bytes) {
  int m = 0, st;
  *bytes = 0;
  if ((st = resolve_method(method, N, &m))) return st;
  if (m != PAULI_XORDIAG || !pauli::tiled_supported(N) || count > 1024) return PAULI_OK;
  const int v = pauli::xordiag_get_variant(N, dtype == PAULI_C64, false, count > 1);
  if (v == pauli::kVariantTiled8 || v == pauli::kVariantTiled16 || v == pauli::kVariantTwoStage)
    *bytes = pauli::tiled_workspace_bytes(N);
  return PAULI_OK;
}

int decompose_checked(const void* G, int N, long long count, int dtype, void* out, int method, cudaStream_t s) {
  int m = 0, st;
  if ((st = resolve_method(method, N, &m))) return st;
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  const bool c64 = dtype == PAULI_C64;
  cudaError_t e = m == PAULI_XORDIAG ? pauli::launch_xordiag(G, N, count, c64, false, 0, out, s)
                                     : pauli::launch_plain_decompose(G, N, count, c64, out, s);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_decompose launch");
  return PAULI_OK;
}

}  // namespace

extern "C" {

const char* pauli_last_error(void) { return g_err.c_str(); }

int pauli_version(void) { return 100; }

void pauli_debug_fail_next_launches(int count) { g_fail_next.store(count > 0 ? count : 0); }

void pauli_debug_stall_next_tiled(void) { pauli::tiled_debug_stall_next(); }

int pauli_decompose(const void* G, int N, int count, int dtype, void* out, int method, void* stream) {
  int st = check_pair(G, "G", N, count, dtype, out, "out");
  if (st) return st;
  return decompose_checked(G, N, count, dtype, out, method, (cudaStream_t)stream);
}

int pauli_decompose_workspace_size(int N, int count, int dtype, int method, size_t* bytes) {
  int st;
  if (!bytes) return fail(PAULI_ERR_NULL, "bytes is NULL");
  *bytes = 0;
  if ((st = check_dtype(dtype))) return st;
  if ((st = check_n(N))) return st;
  if (count < 1) return fail(PAULI_ERR_ARG, "count = %d must be >= 1", count);
  return decompose_workspace_bytes(N, count, dtype, method, bytes);
}

int pauli_decompose_ws(const void* G, int N, int count, int dtype, void* out, int method, void* workspace,
                       size_t workspace_bytes, void* stream) {
  int st = check_pair(G, "G", N, count, dtype, out, "out");
  if (st) return st;
  size_t need = 0;
  if ((st = decompose_workspace_bytes(N, count, dtype, method, &need))) return st;
  if (need) {
    if (!workspace) return fail(PAULI_ERR_NULL, "workspace is NULL (%zu bytes needed)", need);
    if ((st = check_aligned(workspace, 256, "workspace"))) return st;
    if (workspace_bytes < need)
      return fail(PAULI_ERR_ARG, "workspace_bytes = %zu is below the %zu bytes needed", workspace_bytes, need);
    const size_t bytes = (size_t)(1ull << (2 * N)) * (size_t)count * elem_bytes(dtype);
    if (overlaps(workspace, need, G, bytes) || overlaps(workspace, need, out, bytes))
      return fail(PAULI_ERR_ALIAS, "workspace overlaps G or out");
    // this call's status word starts clear (the launch clears the rest of the control block)
    cudaError_t e = cudaMemsetAsync(workspace, 0, pauli::kTiledCtrlBytes, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "pauli_decompose_ws: clearing the workspace");
  }
  pauli::CallerWorkspace guard(pauli::kWorkspaceTiled, workspace, workspace_bytes);
  return decompose_checked(G, N, count, dtype, out, method, (cudaStream_t)stream);
}

int pauli_workspace_status(void* workspace, void* stream) {
  if (!workspace) return fail(PAULI_ERR_NULL, "workspace is NULL");
  const cudaStream_t s = (cudaStream_t)stream;
  int status = 0;
  int* sp = reinterpret_cast<int*>(reinterpret_cast<char*>(workspace) + offsetof(pauli::TiledCtrl, status));
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, sp, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sp, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_workspace_status");
  if (status) return fail(status, "a bounded wait in the tiled decomposition gave up");
  return PAULI_OK;
}

int pauli_release_workspaces(void* stream) {
  cudaError_t e = pauli::stream_workspace_release((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_release_workspaces");
  return PAULI_OK;
}

int pauli_decompose_hermitian(const void* G, int N, int count, int dtype, void* out_re, int method, void* stream) {
  int st = check_real_out(G, N, count, dtype, out_re);
  if (st) return st;
  int m = 0;
  if ((st = resolve_method(method, N, &m))) return st;
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  const bool c64 = dtype == PAULI_C64;
  cudaError_t e = m == PAULI_XORDIAG ? pauli::launch_xordiag_re(G, N, count, c64, out_re, (cudaStream_t)stream)
                                     : pauli::launch_plain_decompose(G, N, count, c64, out_re, (cudaStream_t)stream, true);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_decompose_hermitian launch");
  return PAULI_OK;
}

int pauli_decompose_hermitian_upper(const void* G, int N, int count, int dtype, void* out_re, int method,
                                    void* stream) {
  int st = check_real_out(G, N, count, dtype, out_re);
  if (st) return st;
  if (method != PAULI_AUTO && method != PAULI_PLAIN && method != PAULI_XORDIAG)
    return fail(PAULI_ERR_ARG, "method %d is not a pauli_method", method);
  if (N > 14) return fail(PAULI_ERR_UNSUPPORTED, "pauli_decompose_hermitian_upper is built for N <= 14, not N = %d", N);
  if (method == PAULI_XORDIAG && N < 7)
    return fail(PAULI_ERR_UNSUPPORTED, "the upper-triangle XOR-diagonal kernel starts at N = 7");
  const bool c64 = dtype == PAULI_C64;
  if (N >= 13 && method != PAULI_PLAIN) {  // the two-stage kernel in its upper-triangle mode
    if (count > 1024 || ((uintptr_t)G & 15u))
      return fail(PAULI_ERR_UNSUPPORTED, "the upper-triangle two-stage kernel takes count <= 1024 and 16-byte aligned G");
    if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
    cudaError_t e = pauli::twostage_launch_upper(G, N, count, c64, out_re, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "pauli_decompose_hermitian_upper launch");
    return PAULI_OK;
  }
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  cudaError_t e = (method == PAULI_PLAIN || N < 7)
                      ? pauli::launch_plain_decompose(G, N, count, c64, out_re, (cudaStream_t)stream, true, true)
                      : pauli::launch_xordiag_herm_upper(G, N, count, c64, out_re, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_decompose_hermitian_upper launch");
  return PAULI_OK;
}

int pauli_decompose_real(const void* G_real, int N, int count, int dtype, void* out_re, int method, void* stream) {
  int st;
  if ((st = check_dtype(dtype))) return st;
  if (dtype != PAULI_C128) return fail(PAULI_ERR_UNSUPPORTED, "pauli_decompose_real takes float64 matrices (PAULI_C128)");
  if ((st = check_n(N))) return st;
  if (count < 1) return fail(PAULI_ERR_ARG, "count = %d must be >= 1", count);
  if (!G_real) return fail(PAULI_ERR_NULL, "G_real is NULL");
  if (!out_re) return fail(PAULI_ERR_NULL, "out_re is NULL");
  if ((st = check_aligned(G_real, 8, "G_real"))) return st;
  if ((st = check_aligned(out_re, 8, "out_re"))) return st;
  const unsigned long long per = 1ull << (2 * N);
  if ((unsigned long long)count > (~0ull / 8) / per) return fail(PAULI_ERR_ARG, "count * 4^N overflows");
  const size_t bytes = (size_t)(per * (unsigned long long)count) * 8;
  if (overlaps(G_real, bytes, out_re, bytes)) return fail(PAULI_ERR_ALIAS, "G_real and out_re overlap");
  int m = 0;
  if ((st = resolve_method(method, N, &m))) return st;
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  cudaError_t e = m == PAULI_XORDIAG ? pauli::launch_xordiag_real(G_real, N, count, out_re, (cudaStream_t)stream)
                                     : pauli::launch_plain_decompose_real(G_real, N, count, out_re, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_decompose_real launch");
  return PAULI_OK;
}

int pauli_compose(const void* c, int N, int count, int dtype, void* G_out, int scale_exp, void* stream) {
  int st = check_pair(c, "c", N, count, dtype, G_out, "G_out");
  if (st) return st;
  if (scale_exp < -64 || scale_exp > 64) return fail(PAULI_ERR_ARG, "scale_exp = %d outside [-64, 64]", scale_exp);
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  const bool c64 = dtype == PAULI_C64;
  cudaError_t e = pauli::xordiag_supported(N)
                      ? pauli::launch_xordiag(c, N, count, c64, true, scale_exp, G_out, (cudaStream_t)stream)
                      : pauli::launch_plain_compose(c, N, count, c64, scale_exp, G_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_compose launch");
  return PAULI_OK;
}

int pauli_weighted_norm(const void* c, int N, int count, int dtype, const void* w, void* loss, void* stream) {
  int st;
  if ((st = check_dtype(dtype))) return st;
  if ((st = check_n(N))) return st;
  if (count < 1) return fail(PAULI_ERR_ARG, "count = %d must be >= 1", count);
  if (!c) return fail(PAULI_ERR_NULL, "c is NULL");
  if (!w) return fail(PAULI_ERR_NULL, "w is NULL");
  if (!loss) return fail(PAULI_ERR_NULL, "loss is NULL");
  const size_t es = elem_bytes(dtype), rs = es / 2;
  if ((st = check_aligned(c, es, "c"))) return st;
  if ((st = check_aligned(w, rs, "w"))) return st;
  if ((st = check_aligned(loss, rs, "loss"))) return st;
  const size_t per = (size_t)1 << (2 * N);
  if ((unsigned long long)count > (~0ull / es) / per) return fail(PAULI_ERR_ARG, "count * 4^N overflows");
  if (overlaps(loss, rs, c, per * (size_t)count * es) || overlaps(loss, rs, w, per * rs))
    return fail(PAULI_ERR_ALIAS, "loss overlaps c or w");
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  cudaError_t e = pauli::launch_weighted_norm(c, N, count, dtype == PAULI_C64, w, loss, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_weighted_norm launch");
  return PAULI_OK;
}

int pauli_weighted_norm_grad(const void* c, int N, int count, int dtype, const void* w, const void* g, void* grad_c,
                             void* stream) {
  int st;
  if ((st = check_dtype(dtype))) return st;
  if ((st = check_n(N))) return st;
  if (count < 1) return fail(PAULI_ERR_ARG, "count = %d must be >= 1", count);
  if (!c) return fail(PAULI_ERR_NULL, "c is NULL");
  if (!w) return fail(PAULI_ERR_NULL, "w is NULL");
  if (!grad_c) return fail(PAULI_ERR_NULL, "grad_c is NULL");
  const size_t es = elem_bytes(dtype), rs = es / 2;
  if ((st = check_aligned(c, es, "c"))) return st;
  if ((st = check_aligned(grad_c, es, "grad_c"))) return st;
  if ((st = check_aligned(w, rs, "w"))) return st;
  if (g && (st = check_aligned(g, rs, "g"))) return st;
  const size_t per = (size_t)1 << (2 * N);
  if ((unsigned long long)count > (~0ull / es) / per) return fail(PAULI_ERR_ARG, "count * 4^N overflows");
  const size_t bytes = per * (size_t)count * es;
  if (grad_c != c && overlaps(grad_c, bytes, c, bytes))
    return fail(PAULI_ERR_ALIAS, "grad_c overlaps c without being equal to it");
  if (overlaps(grad_c, bytes, w, per * rs) || (g && overlaps(grad_c, bytes, g, rs)))
    return fail(PAULI_ERR_ALIAS, "grad_c overlaps w or g");
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  cudaError_t e =
      pauli::launch_weighted_norm_grad(c, N, count, dtype == PAULI_C64, w, g, grad_c, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_weighted_norm_grad launch");
  return PAULI_OK;
}

int pauli_decompose_weighted_norm(const void* G, int N, int count, int dtype, void* out, const void* w, void* loss,
                                  int method, void* stream) {
  int st = check_pair(G, "G", N, count, dtype, out, "out");
  if (st) return st;
  if (!w) return fail(PAULI_ERR_NULL, "w is NULL");
  if (!loss) return fail(PAULI_ERR_NULL, "loss is NULL");
  const size_t es = elem_bytes(dtype), rs = es / 2;
  if ((st = check_aligned(w, rs, "w"))) return st;
  if ((st = check_aligned(loss, rs, "loss"))) return st;
  const size_t per = (size_t)1 << (2 * N), bytes = per * (size_t)count * es;
  if (overlaps(out, bytes, w, per * rs) || overlaps(loss, rs, out, bytes) || overlaps(loss, rs, G, bytes) ||
      overlaps(loss, rs, w, per * rs))
    return fail(PAULI_ERR_ALIAS, "out, w and loss must not overlap each other or G");
  int m = 0;
  if ((st = resolve_method(method, N, &m))) return st;
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  cudaError_t e = pauli::launch_decompose_norm(G, N, count, dtype == PAULI_C64, out, w, loss,
                                               m == PAULI_PLAIN ? 1 : 2, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_decompose_weighted_norm launch");
  return PAULI_OK;
}

int pauli_compose_weighted(const void* c, int N, int count, int dtype, const void* w, const void* g, void* G_out,
                           int scale_exp, void* stream) {
  int st = check_pair(c, "c", N, count, dtype, G_out, "G_out");
  if (st) return st;
  if (scale_exp < -64 || scale_exp > 64) return fail(PAULI_ERR_ARG, "scale_exp = %d outside [-64, 64]", scale_exp);
  if (!w) return fail(PAULI_ERR_NULL, "w is NULL");
  const size_t es = elem_bytes(dtype), rs = es / 2;
  if ((st = check_aligned(w, rs, "w"))) return st;
  if (g && (st = check_aligned(g, rs, "g"))) return st;
  const size_t per = (size_t)1 << (2 * N), bytes = per * (size_t)count * es;
  if (overlaps(G_out, bytes, w, per * rs) || (g && overlaps(G_out, bytes, g, rs)))
    return fail(PAULI_ERR_ALIAS, "G_out overlaps w or g");
  if (N > 12) return fail(PAULI_ERR_UNSUPPORTED, "pauli_compose_weighted is built for N <= 12, not N = %d", N);
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  cudaError_t e =
      pauli::launch_compose_weighted(c, N, count, dtype == PAULI_C64, w, g, scale_exp, G_out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_compose_weighted launch");
  return PAULI_OK;
}

int pauli_set_variant(int N, int dtype, int op, int variant) {
  int st;
  if ((st = check_dtype(dtype))) return st;
  if ((st = check_n(N))) return st;
  if (op < 0 || op > 3)
    return fail(PAULI_ERR_ARG, "op = %d is not 0/1 (decompose/compose) or 2/3 (the same for batches)", op);
  const bool compose = op & 1, batched = op >= 2;
  if (variant != PAULI_VARIANT_DEFAULT && !pauli::xordiag_variant_supported(variant, N, compose))
    return fail(PAULI_ERR_UNSUPPORTED, "variant %d has no %s kernel for N = %d", variant,
                compose ? "compose" : "decompose", N);
  pauli::xordiag_set_variant(N, dtype == PAULI_C64, compose, batched, variant);
  return PAULI_OK;
}

int pauli_stream_status(void* stream) {
  int status = 0;
  cudaError_t e = pauli::tiled_stream_status((cudaStream_t)stream, &status);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_stream_status");
  if (status) return fail(status, "a bounded wait in the tiled decomposition gave up");
  return PAULI_OK;
}

int pauli_get_variant(int N, int dtype, int op) {
  if (check_dtype(dtype) || check_n(N) || op < 0 || op > 3) return 0;
  return pauli::xordiag_get_variant(N, dtype == PAULI_C64, op & 1, op >= 2);
}

int pauli_coeffs_at(const void* G, int N, int dtype, const uint64_t* idx, int64_t k, void* out, void* stream) {
  int st;
  if ((st = check_dtype(dtype))) return st;
  if ((st = check_n(N))) return st;
  if (k < 0) return fail(PAULI_ERR_ARG, "k = %lld must be >= 0", (long long)k);
  if (k == 0) return PAULI_OK;
  if (!G) return fail(PAULI_ERR_NULL, "G is NULL");
  if (!idx) return fail(PAULI_ERR_NULL, "idx is NULL");
  if (!out) return fail(PAULI_ERR_NULL, "out is NULL");
  const size_t es = elem_bytes(dtype);
  if ((st = check_aligned(G, es, "G"))) return st;
  if ((st = check_aligned(out, es, "out"))) return st;
  if ((st = check_aligned(idx, 8, "idx"))) return st;
  const size_t gbytes = (size_t)(1ull << (2 * N)) * es, obytes = (size_t)k * es;
  if (overlaps(G, gbytes, out, obytes) || overlaps(idx, (size_t)k * 8, out, obytes))
    return fail(PAULI_ERR_ALIAS, "out overlaps G or idx");
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  cudaError_t e = pauli::launch_coeffs_at(G, N, dtype == PAULI_C64, idx, k, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_coeffs_at launch");
  return PAULI_OK;
}

int pauli_decompose_list(const void* const* G_list, const int* N_list, int batch, int dtype, void* const* out_list,
                         int method, void* stream) {
  if (batch < 0) return fail(PAULI_ERR_ARG, "batch = %d must be >= 0", batch);
  if (batch == 0) return PAULI_OK;
  if (!G_list || !N_list || !out_list) return fail(PAULI_ERR_NULL, "G_list, N_list and out_list must not be NULL");
  for (int b = 0; b < batch; ++b) {
    int st = check_pair(G_list[b], "G_list[b]", N_list[b], 1, dtype, out_list[b], "out_list[b]");
    if (st) return fail(st, "entry %d: %s", b, g_err.c_str());
  }
  for (int b = 0; b < batch; ++b) {
    int st = decompose_checked(G_list[b], N_list[b], 1, dtype, out_list[b], method, (cudaStream_t)stream);
    if (st) return st;
  }
  return PAULI_OK;
}

int pauli_compose_batched(const void* const* c_list, const int* N_list, int batch, int dtype, void* const* G_out_list,
                          int scale_exp, void* stream) {
  int st;
  if ((st = check_dtype(dtype))) return st;
  if (batch < 0) return fail(PAULI_ERR_ARG, "batch = %d must be >= 0", batch);
  if (batch == 0) return PAULI_OK;
  if (!c_list || !N_list || !G_out_list) return fail(PAULI_ERR_NULL, "c_list, N_list and G_out_list must not be NULL");
  if (scale_exp < -64 || scale_exp > 64) return fail(PAULI_ERR_ARG, "scale_exp = %d outside [-64, 64]", scale_exp);
  const int nmax = pauli::compose_batched_max_n();
  for (int b = 0; b < batch; ++b) {
    if (N_list[b] < 1 || N_list[b] > nmax)
      return fail(PAULI_ERR_ARG, "N_list[%d] = %d outside [1, %d]", b, N_list[b], nmax);
    st = check_pair(c_list[b], "c_list[b]", N_list[b], 1, dtype, G_out_list[b], "G_out_list[b]");
    if (st) return fail(st, "entry %d: %s", b, g_err.c_str());
  }
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  cudaError_t e = pauli::launch_compose_batched(c_list, N_list, batch, dtype == PAULI_C64, G_out_list, scale_exp,
                                                (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_compose_batched launch");
  return PAULI_OK;
}

int pauli_xhi_layout(const void* G, int N, int k, int x_hi, int dtype, void* L, void* stream) {
  int st;
  if ((st = check_dtype(dtype))) return st;
  if ((st = check_n(N))) return st;
  if (k < 0 || k >= N) return fail(PAULI_ERR_ARG, "k = %d outside [0, N - 1] for N = %d", k, N);
  if (x_hi < 0 || x_hi >= (1 << k)) return fail(PAULI_ERR_ARG, "x_hi = %d outside [0, 2^k) for k = %d", x_hi, k);
  if (!G) return fail(PAULI_ERR_NULL, "G is NULL");
  if (!L) return fail(PAULI_ERR_NULL, "L is NULL");
  const size_t es = elem_bytes(dtype);
  if ((st = check_aligned(G, es, "G"))) return st;
  if ((st = check_aligned(L, es, "L"))) return st;
  const size_t full = ((size_t)1 << (2 * N)) * es;
  if (overlaps(G, full, L, full >> k)) return fail(PAULI_ERR_ALIAS, "G and L overlap");
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  cudaError_t e = pauli::xhi_layout(G, N, k, (uint32_t)x_hi, es, L, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_xhi_layout copies");
  return PAULI_OK;
}

int pauli_decompose_xhi(const void* L, int N, int k, int x_hi, int dtype, void* out, int method, void* stream) {
  int st;
  if ((st = check_dtype(dtype))) return st;
  if ((st = check_n(N))) return st;
  if (k < 0 || k >= N) return fail(PAULI_ERR_ARG, "k = %d outside [0, N - 1] for N = %d", k, N);
  if (x_hi < 0 || x_hi >= (1 << k)) return fail(PAULI_ERR_ARG, "x_hi = %d outside [0, 2^k) for k = %d", x_hi, k);
  // the shard is 2^k stacked (N - k)-qubit blocks in, as many coefficients out
  if ((st = check_pair(L, "L", N - k, 1ll << k, dtype, out, "out"))) return st;
  int m = 0;
  if ((st = resolve_method(method, N - k, &m))) return st;
  if (m == PAULI_XORDIAG && N >= 12 && N <= 14 && N - k >= 6 && !((uintptr_t)L & 15u)) {
    // the whole shard in one two-stage launch
    if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
    cudaError_t e = pauli::twostage_launch_xhi(L, N, k, (uint32_t)x_hi, dtype == PAULI_C64, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "pauli_decompose_xhi launch");
    return PAULI_OK;
  }
  if ((st = decompose_checked(L, N - k, 1ll << k, dtype, out, method, (cudaStream_t)stream))) return st;
  cudaError_t e = pauli::launch_xhi_combine(out, N, k, (uint32_t)x_hi, dtype == PAULI_C64, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_decompose_xhi combine launch");
  return PAULI_OK;
}

int pauli_decompose_batch_static(const void* const* G_list, const int* N_list, int batch, int dtype,
                                 void* const* out_list, void* stream) {
  int st;
  if ((st = check_dtype(dtype))) return st;
  if (batch < 1 || batch > pauli::static_batch_max())
    return fail(PAULI_ERR_ARG, "batch = %d outside [1, %d] (the static scratch holds at most %d matrices)", batch,
                pauli::static_batch_max(), pauli::static_batch_max());
  if (!G_list || !N_list || !out_list) return fail(PAULI_ERR_NULL, "G_list, N_list and out_list must not be NULL");
  for (int b = 0; b < batch; ++b) {
    if (N_list[b] < 1 || N_list[b] > 10) return fail(PAULI_ERR_ARG, "N_list[%d] = %d outside [1, 10]", b, N_list[b]);
    st = check_pair(G_list[b], "G_list[b]", N_list[b], 1, dtype, out_list[b], "out_list[b]");
    if (st) return fail(st, "entry %d: %s", b, g_err.c_str());
  }
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  const char* what = "";
  cudaError_t ce = cudaSuccess;
  st = pauli::static_batch_launch(G_list, N_list, batch, dtype == PAULI_C64, out_list, (cudaStream_t)stream, &what,
                                  &ce);
  if (st == PAULI_ERR_CUDA) return cuda_fail(ce, what);
  if (st) return fail(st, "%s", what);
  return PAULI_OK;
}

int pauli_decompose_host(const void* G_host, int N, int count, int dtype, void* out_host, void* G_dev, void* out_dev,
                         int method, void* stream) {
  int st = check_pair(G_dev, "G_dev", N, count, dtype, out_dev, "out_dev");
  if (st) return st;
  if (!G_host) return fail(PAULI_ERR_NULL, "G_host is NULL");
  if (!out_host) return fail(PAULI_ERR_NULL, "out_host is NULL");
  const size_t bytes = (size_t)((1ull << (2 * N)) * (unsigned long long)count) * elem_bytes(dtype);
  if (overlaps(G_host, bytes, out_host, bytes)) return fail(PAULI_ERR_ALIAS, "G_host and out_host overlap");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(G_dev, G_host, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_decompose_host: copy to device");
  if ((st = decompose_checked(G_dev, N, count, dtype, out_dev, method, s))) return st;
  e = cudaMemcpyAsync(out_host, out_dev, bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_decompose_host: copy to host");
  return PAULI_OK;
}

int pauli_decompose_host_stream(const void* const* G_host_list, void* const* out_host_list, int n_mats, int N,
                                int dtype, void* const* G_dev, void* const* out_dev, int method, void* stream) {
  if (!G_host_list || !out_host_list) return fail(PAULI_ERR_NULL, "G_host_list and out_host_list must not be NULL");
  if (!G_dev || !out_dev) return fail(PAULI_ERR_NULL, "G_dev and out_dev must not be NULL");
  if (n_mats < 1) return fail(PAULI_ERR_ARG, "n_mats = %d must be >= 1", n_mats);
  int st;
  for (int b = 0; b < 2; ++b)
    if ((st = check_pair(G_dev[b], "G_dev[b]", N, 1, dtype, out_dev[b], "out_dev[b]"))) return st;
  const size_t bytes = (size_t)(1ull << (2 * N)) * elem_bytes(dtype);
  const void* bufs[4] = {G_dev[0], G_dev[1], out_dev[0], out_dev[1]};
  for (int i = 0; i < 4; ++i)
    for (int j = i + 1; j < 4; ++j)
      if (overlaps(bufs[i], bytes, bufs[j], bytes)) return fail(PAULI_ERR_ALIAS, "the four device buffers overlap");
  for (int k = 0; k < n_mats; ++k) {
    if (!G_host_list[k] || !out_host_list[k]) return fail(PAULI_ERR_NULL, "host buffer %d is NULL", k);
    if (overlaps(G_host_list[k], bytes, out_host_list[k], bytes))
      return fail(PAULI_ERR_ALIAS, "G_host_list[%d] and out_host_list[%d] overlap", k, k);
  }
  int m = 0;
  if ((st = resolve_method(method, N, &m))) return st;
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  HostPipe* hp = nullptr;
  cudaError_t e = host_pipe(&hp);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_decompose_host_stream: streams");
  std::lock_guard<std::mutex> lock(hp->mutex);
  const cudaStream_t user = (cudaStream_t)stream;
  // the pipeline starts after earlier work on the caller's stream
  if ((e = cudaEventRecord(hp->start, user)) != cudaSuccess) return cuda_fail(e, "pauli_decompose_host_stream");
  for (cudaStream_t s : {hp->in, hp->comp, hp->out})
    if ((e = cudaStreamWaitEvent(s, hp->start, 0)) != cudaSuccess) return cuda_fail(e, "pauli_decompose_host_stream");
  for (int k = 0; k < n_mats; ++k) {
    const int b = k & 1;
    // copy in: buffer b is free once the decomposition of matrix k - 2 has read it
    if (k >= 2 && (e = cudaStreamWaitEvent(hp->in, hp->comp_done[b], 0)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(G_dev[b], G_host_list[k], bytes, cudaMemcpyHostToDevice, hp->in)) != cudaSuccess) break;
    if ((e = cudaEventRecord(hp->in_done[b], hp->in)) != cudaSuccess) break;
    // decompose: needs matrix k in, and out_dev[b] copied out for matrix k - 2
    if ((e = cudaStreamWaitEvent(hp->comp, hp->in_done[b], 0)) != cudaSuccess) break;
    if (k >= 2 && (e = cudaStreamWaitEvent(hp->comp, hp->out_done[b], 0)) != cudaSuccess) break;
    if ((st = decompose_checked(G_dev[b], N, 1, dtype, out_dev[b], m, hp->comp))) return st;
    if ((e = cudaEventRecord(hp->comp_done[b], hp->comp)) != cudaSuccess) break;
    // copy out
    if ((e = cudaStreamWaitEvent(hp->out, hp->comp_done[b], 0)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(out_host_list[k], out_dev[b], bytes, cudaMemcpyDeviceToHost, hp->out)) != cudaSuccess)
      break;
    if ((e = cudaEventRecord(hp->out_done[b], hp->out)) != cudaSuccess) break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "pauli_decompose_host_stream: enqueue");
  // later work on the caller's stream waits for the last copy out (which follows everything else)
  if ((e = cudaEventRecord(hp->end, hp->out)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(user, hp->end, 0)) != cudaSuccess)
    return cuda_fail(e, "pauli_decompose_host_stream: join");
  return PAULI_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------ plans --
struct pauli_plan {
  std::vector<int> Ns;
  bool herm = false;  // Hermitian matrices read from the upper triangle, real outputs
  int dtype = PAULI_C128;
  int UB = 13;
  int blocks_per_sm = 0;
  int n_items = 0;
  pauli::PlanItem* d_items = nullptr;
  pauli::PlanMat* d_mats = nullptr;
  pauli::PlanCtrl* d_ctrl = nullptr;
  bool bound = false;
  cudaStream_t last = nullptr;
  cudaStream_t capture = nullptr;
  cudaGraphExec_t graph = nullptr;
};

namespace {

void plan_free(pauli_plan* p) {
  if (!p) return;
  if (p->graph) cudaGraphExecDestroy(p->graph);
  if (p->capture) cudaStreamDestroy(p->capture);
  cudaFree(p->d_items);
  cudaFree(p->d_mats);
  cudaFree(p->d_ctrl);
  delete p;
}

int plan_enqueue(pauli_plan* p, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(p->d_ctrl, 0, 2 * sizeof(int), s);  // counter, status
  if (e != cudaSuccess) return cuda_fail(e, "plan reset");
  e = pauli::launch_plan(p->d_items, p->n_items, p->d_mats, p->d_ctrl, p->dtype == PAULI_C64, p->UB, p->blocks_per_sm,
                         s, 0, p->herm);
  if (e != cudaSuccess) return cuda_fail(e, "plan launch");
  return PAULI_OK;
}

int plan_create(const int* N_list, int batch, int dtype, int threads_per_block, int blocks_per_sm, bool herm,
                pauli_plan** plan) {
  int st;
  if (!plan) return fail(PAULI_ERR_NULL, "plan is NULL");
  *plan = nullptr;
  if ((st = check_dtype(dtype))) return st;
  if (batch < 1) return fail(PAULI_ERR_ARG, "batch = %d must be >= 1", batch);
  if (!N_list) return fail(PAULI_ERR_NULL, "N_list is NULL");
  if (threads_per_block != 0 && threads_per_block != 256 && threads_per_block != 512)
    return fail(PAULI_ERR_ARG, "threads_per_block = %d is not 0, 256 or 512", threads_per_block);
  if (blocks_per_sm < 0) return fail(PAULI_ERR_ARG, "blocks_per_sm = %d must be >= 0", blocks_per_sm);
  for (int b = 0; b < batch; ++b)
    if (N_list[b] < 1 || N_list[b] > 10) return fail(PAULI_ERR_ARG, "N_list[%d] = %d outside [1, 10]", b, N_list[b]);
  pauli_plan* p = new (std::nothrow) pauli_plan;
  if (!p) return fail(PAULI_ERR_NOMEM, "plan allocation failed");
  p->Ns.assign(N_list, N_list + batch);
  p->herm = herm;
  p->dtype = dtype;
  p->UB = threads_per_block == 256 ? 12 : 13;
  p->blocks_per_sm = blocks_per_sm;
  // work list: one item per unit (or per small matrix), largest N first
  std::vector<pauli::PlanItem> items;
  std::vector<int> order(batch);
  for (int b = 0; b < batch; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return N_list[a] > N_list[b]; });
  for (int b : order) {
    const unsigned units = pauli::plan_units(N_list[b], p->UB, herm);
    for (unsigned u = 0; u < units; ++u) items.push_back(pauli::PlanItem{(uint32_t)b, u});
  }
  p->n_items = (int)items.size();
  cudaError_t e;
  if ((e = cudaMalloc(&p->d_items, items.size() * sizeof(pauli::PlanItem))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_mats, batch * sizeof(pauli::PlanMat))) != cudaSuccess ||
      (e = cudaMalloc(&p->d_ctrl, sizeof(pauli::PlanCtrl))) != cudaSuccess) {
    plan_free(p);
    return fail(PAULI_ERR_NOMEM, "plan device allocation failed: %s", cudaGetErrorString(e));
  }
  e = cudaMemcpy(p->d_items, items.data(), items.size() * sizeof(pauli::PlanItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(p->d_ctrl, 0, sizeof(pauli::PlanCtrl));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->capture, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    plan_free(p);
    return cuda_fail(e, "pauli_plan_create");
  }
  *plan = p;
  return PAULI_OK;
}

}  // namespace

extern "C" {

int pauli_plan_create(const int* N_list, int batch, int dtype, int threads_per_block, int blocks_per_sm,
                      pauli_plan** plan) {
  return plan_create(N_list, batch, dtype, threads_per_block, blocks_per_sm, false, plan);
}

int pauli_plan_create_hermitian(const int* N_list, int batch, int dtype, int threads_per_block, int blocks_per_sm,
                                pauli_plan** plan) {
  return plan_create(N_list, batch, dtype, threads_per_block, blocks_per_sm, true, plan);
}

int pauli_plan_bind(pauli_plan* p, const void* const* G_list, void* const* out_list) {
  if (!p) return fail(PAULI_ERR_NULL, "plan is NULL");
  if (!G_list || !out_list) return fail(PAULI_ERR_NULL, "G_list and out_list must not be NULL");
  std::vector<pauli::PlanMat> mats(p->Ns.size());
  for (size_t b = 0; b < p->Ns.size(); ++b) {
    int st = p->herm ? check_real_out(G_list[b], p->Ns[b], 1, p->dtype, out_list[b])
                     : check_pair(G_list[b], "G_list[b]", p->Ns[b], 1, p->dtype, out_list[b], "out_list[b]");
    if (st) return fail(st, "entry %zu: %s", b, g_err.c_str());
    mats[b] = pauli::PlanMat{G_list[b], out_list[b], p->Ns[b], 0};  // items list in use: first unused
  }
  cudaError_t e = cudaMemcpy(p->d_mats, mats.data(), mats.size() * sizeof(pauli::PlanMat), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_plan_bind");
  p->bound = true;
  return PAULI_OK;
}

int pauli_plan_execute(pauli_plan* p, void* stream) {
  if (!p) return fail(PAULI_ERR_NULL, "plan is NULL");
  if (!p->bound) return fail(PAULI_ERR_ARG, "plan has no bound buffers (call pauli_plan_bind)");
  if (take_injected_failure()) return fail(PAULI_ERR_CUDA, "injected launch failure (test hook)");
  p->last = (cudaStream_t)stream;
  return plan_enqueue(p, p->last);
}

int pauli_plan_graph_launch(pauli_plan* p, void* stream) {
  if (!p) return fail(PAULI_ERR_NULL, "plan is NULL");
  if (!p->bound) return fail(PAULI_ERR_ARG, "plan has no bound buffers (call pauli_plan_bind)");
  if (!p->graph) {
    // capture on the plan's own stream (the caller's may be the legacy default stream)
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(p->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "plan capture");
    int st = plan_enqueue(p, p->capture);
    e = cudaStreamEndCapture(p->capture, &g);
    if (st) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "plan capture end");
    e = cudaGraphInstantiate(&p->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      p->graph = nullptr;
      return cuda_fail(e, "plan graph instantiate");
    }
  }
  p->last = (cudaStream_t)stream;
  cudaError_t e = cudaGraphLaunch(p->graph, p->last);
  if (e != cudaSuccess) return cuda_fail(e, "plan graph launch");
  return PAULI_OK;
}

int pauli_plan_status(pauli_plan* p) {
  if (!p) return fail(PAULI_ERR_NULL, "plan is NULL");
  cudaError_t e = cudaStreamSynchronize(p->last);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_plan_status");
  int status = 0;
  e = cudaMemcpy(&status, &p->d_ctrl->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_plan_status");
  if (status) return fail(status, "a bounded wait in the plan kernel gave up");
  return PAULI_OK;
}

int pauli_plan_set_stall(pauli_plan* p, int stall) {
  if (!p) return fail(PAULI_ERR_NULL, "plan is NULL");
  const int v = stall ? 1 : 0;
  cudaError_t e = cudaMemcpy(&p->d_ctrl->stall, &v, sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "pauli_plan_set_stall");
  return PAULI_OK;
}

void pauli_plan_destroy(pauli_plan* p) { plan_free(p); }

}  // extern "C"

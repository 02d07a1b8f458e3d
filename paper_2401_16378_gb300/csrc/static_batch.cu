// static_batch.cu -- batched decomposition that allocates nothing.
//
// Some callers cannot allocate device memory: code that runs where the caching allocator
// it shares memory with must not be re-entered, code whose memory budget is fixed up front,
// or code running while another component holds the allocator. pauli_plan_create needs
// cudaMalloc for its work list and control block; pauli_decompose_batch_static does the same
// one-launch batched decomposition with that state in a fixed-size array in device global
// memory that is part of the library image (every GPU that loads the library holds it until
// the process exits): a control block (work counter, status) and a table of at most
// kStaticMaxBatch matrices. The work items are not stored; the kernel finds the matrix of
// item i by binary search over the table's running item counts.
//
// The table reaches the array through a small kernel that receives it by value, as a kernel
// parameter (24 KiB at most, inside the 32 KiB parameter limit), and also clears the control
// block. Kernel parameters are copied when the launch is enqueued, so the call returns without
// waiting for the GPU, the caller's host arrays may be reused at once, and a graph that captured
// a call replays that call's own table.
//
// All calls share the array and it keeps the last call's contents. Calls whose kernels overlap
// on the GPU (different streams, or different threads without ordering) race on the array and
// must be serialised by the caller. The first call on each device looks up the array's device
// address with cudaGetSymbolAddress (with that device current) and caches it; make that first
// call before capturing the stream into a CUDA graph.
#include <mutex>

#include "pauli.h"
#include "plan_internal.h"

namespace pauli {
namespace {

constexpr int kStaticMaxBatch = 1024;

struct StaticScratch {
  PlanCtrl ctrl;
  int pad[4];
  PlanMat mats[kStaticMaxBatch];
};
constexpr size_t kStaticScratchBytes = sizeof(StaticScratch);  // 24,608 bytes

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
StaticScratch* g_scratch_ptr[kMaxDevices] = {};

// Device address of the array for the current device (looked up once per device).
cudaError_t scratch_for_current_device(StaticScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = reinterpret_cast<StaticScratch*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// The matrix table as a kernel parameter.
struct StaticTableArgs {
  PlanMat mats[kStaticMaxBatch];
};
static_assert(sizeof(StaticTableArgs) + 16 <= 32764, "the table fits the kernel parameter limit");

// Copies the table into the array and clears the control block (one thread per entry).
__global__ void static_table_store(const __grid_constant__ StaticTableArgs a, int batch, StaticScratch* s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < batch) s->mats[i] = a.mats[i];
  if (i == 0) s->ctrl = PlanCtrl{0, 0, 0, 0};
}

// Host staging of the table, one per thread (its contents are copied at the launch).
thread_local StaticTableArgs t_args;
thread_local int t_order[kStaticMaxBatch];

}  // namespace

int static_batch_max() { return kStaticMaxBatch; }

// Returns a pauli_status; *what receives a short reason on failure.
int static_batch_launch(const void* const* G_list, const int* N_list, int batch, bool c64, void* const* out_list,
                        cudaStream_t s, const char** what, cudaError_t* cuda_err) {
  *cuda_err = cudaSuccess;
  if (batch < 1 || batch > kStaticMaxBatch) {
    *what = "batch must be between 1 and the static maximum (1024)";
    return PAULI_ERR_ARG;
  }
  // largest N first (stable counting sort over N in 1..10), running item counts
  int n = 0;
  for (int N = 10; N >= 1; --N)
    for (int b = 0; b < batch; ++b)
      if (N_list[b] == N) t_order[n++] = b;
  if (n != batch) {
    *what = "every N must be between 1 and 10";
    return PAULI_ERR_ARG;
  }
  const int nmin = plan_min_unit_n(13);
  long long items = 0;
  for (int i = 0; i < batch; ++i) {
    const int b = t_order[i], N = N_list[b];
    t_args.mats[i] = PlanMat{G_list[b], out_list[b], N, (int)items};
    items += N >= nmin ? (long long)((1ull << (2 * N)) >> 13) : 1ll;
  }
  StaticScratch* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e == cudaSuccess) {
    static_table_store<<<(batch + 255) / 256, 256, 0, s>>>(t_args, batch, scratch);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_plan(nullptr, (int)items, scratch->mats, &scratch->ctrl, c64, 13, 0, s, batch);
  if (e != cudaSuccess) {
    *what = "static batch launch";
    *cuda_err = e;
    return PAULI_ERR_CUDA;
  }
  return PAULI_OK;
}

}  // namespace pauli

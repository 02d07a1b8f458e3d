// compose_batched.cu -- host side of the batched composition: the matrix table and its launches.
#include <vector>

#include "compose_batched.cuh"
#include "kernels.h"

namespace pauli {

cudaError_t compose_batched_c128(const cb::ComposeTable&, int, int, int, cudaStream_t);
cudaError_t compose_batched_c64(const cb::ComposeTable&, int, int, int, cudaStream_t);

namespace {
thread_local cb::ComposeTable t_table;  // host staging; its contents are copied at each launch
}  // namespace

int compose_batched_max_n() { return cb::kMaxN; }

// One launch per 1024 matrices, each with its slice of the batch sorted by decreasing N.
cudaError_t launch_compose_batched(const void* const* c_list, const int* N_list, int batch, bool c64,
                                   void* const* G_list, int scale_exp, cudaStream_t s) {
  std::vector<int> order;
  order.reserve(batch);
  for (int N = cb::kMaxN; N >= 1; --N)
    for (int b = 0; b < batch; ++b)
      if (N_list[b] == N) order.push_back(b);
  if ((int)order.size() != batch) return cudaErrorInvalidValue;
  for (int start = 0; start < batch; start += cb::kMaxTable) {
    const int n = batch - start < cb::kMaxTable ? batch - start : cb::kMaxTable;
    long long items = 0;
    for (int i = 0; i < n; ++i) {
      const int b = order[start + i], N = N_list[b];
      t_table.mats[i] = PlanMat{c_list[b], G_list[b], N, (int)items};
      items += cb::items_of(N);
    }
    if (items > 0x7FFFFFFFll) return cudaErrorInvalidValue;
    const cudaError_t e = c64 ? compose_batched_c64(t_table, n, (int)items, scale_exp, s)
                              : compose_batched_c128(t_table, n, (int)items, scale_exp, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pauli

// plan_internal.h -- device-side records of a plan (shared by plan.cu and capi.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pauli {

struct PlanMat {
  const void* in;
  void* out;
  int N;
  int first;  // index of this matrix's first work item (used when there is no item list)
};
struct PlanItem {
  uint32_t mat;   // index into the matrix table
  uint32_t unit;  // unit index within the matrix (0 for a small matrix)
};
struct PlanCtrl {
  int counter;  // next work item
  int status;   // pauli_status of the last execution
  int stall;    // test hook: wait on `never` before starting
  int never;    // never set
};

// Smallest N processed as XOR-diagonal units (smaller matrices are one item each).
__host__ __device__ inline int plan_min_unit_n(int UB) { return UB == 12 ? 6 : 7; }
// items == nullptr: the work list is given by mats[b].first over `batch` matrices.
cudaError_t launch_plan(const PlanItem* items, int n_items, const PlanMat* mats, PlanCtrl* ctrl, bool c64, int UB,
                        int blocks_per_sm, cudaStream_t s, int batch = 0);

}  // namespace pauli

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
// The same for Hermitian plans. An upper-triangle unit holds 2^(UB - N + 1) classes, at most all
// 2^N; with 4096-element units N = 6 is one full-row unit (whole matrix), one item.
__host__ __device__ inline int plan_min_herm_n(int UB) { return UB == 12 ? 6 : 7; }
// Work units of an N-qubit matrix in a plan (1 below the threshold).
__host__ __device__ inline unsigned plan_units(int N, int UB, bool herm) {
  if (N < (herm ? plan_min_herm_n(UB) : plan_min_unit_n(UB))) return 1u;
  if (!herm) return (unsigned)((1ull << (2 * N)) >> UB);
  if (2 * N <= UB) return 1u;  // one full-row unit holds the whole matrix (N = 6, UB = 12)
  return (unsigned)((1ull << N) >> (UB - N + 1));
}
// items == nullptr: the work list is given by mats[b].first over `batch` matrices.
cudaError_t launch_plan(const PlanItem* items, int n_items, const PlanMat* mats, PlanCtrl* ctrl, bool c64, int UB,
                        int blocks_per_sm, cudaStream_t s, int batch = 0, bool herm = false);

}  // namespace pauli

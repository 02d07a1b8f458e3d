// plan_u12_c64.cu -- plan kernel instantiation: 256-thread CTAs, c64.
#include "plan_kernels.cuh"

namespace pauli {

cudaError_t plan_u12_c64(const PlanItem* items, int n_items, const PlanMat* mats, PlanCtrl* ctrl, int blocks_per_sm,
                  cudaStream_t s, int batch) {
  return pk::launch_plan_t<12, xd::ArC64>(items, n_items, mats, ctrl, blocks_per_sm, s, batch);
}

}  // namespace pauli

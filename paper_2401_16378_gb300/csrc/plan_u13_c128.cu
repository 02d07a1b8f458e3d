// plan_u13_c128.cu -- plan kernel instantiation: 512-thread CTAs, c128.
#include "plan_kernels.cuh"

namespace pauli {

cudaError_t plan_u13_c128(const PlanItem* items, int n_items, const PlanMat* mats, PlanCtrl* ctrl, int blocks_per_sm,
                  cudaStream_t s, int batch) {
  return pk::launch_plan_t<13, xd::ArC128>(items, n_items, mats, ctrl, blocks_per_sm, s, batch);
}

}  // namespace pauli

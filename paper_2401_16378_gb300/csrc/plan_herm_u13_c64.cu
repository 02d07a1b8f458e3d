// plan_herm_u13_c64.cu -- Hermitian plan kernel instantiation: 512-thread CTAs, c64,
// matrices read from their upper triangle, real coefficients.
#include "plan_kernels.cuh"

namespace pauli {

cudaError_t plan_herm_u13_c64(const PlanItem* items, int n_items, const PlanMat* mats, PlanCtrl* ctrl,
                                int blocks_per_sm, cudaStream_t s, int batch) {
  return pk::launch_plan_t<13, xd::ReOut<xd::ArC64>, true>(items, n_items, mats, ctrl, blocks_per_sm, s, batch);
}

}  // namespace pauli

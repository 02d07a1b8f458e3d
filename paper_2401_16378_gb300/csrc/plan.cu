// plan.cu -- dispatch of the persistent batched plan kernel (see plan_kernels.cuh).
#include "kernels.h"
#include "plan_internal.h"

namespace pauli {

cudaError_t plan_u12_c128(const PlanItem*, int, const PlanMat*, PlanCtrl*, int, cudaStream_t, int);
cudaError_t plan_u12_c64(const PlanItem*, int, const PlanMat*, PlanCtrl*, int, cudaStream_t, int);
cudaError_t plan_u13_c128(const PlanItem*, int, const PlanMat*, PlanCtrl*, int, cudaStream_t, int);
cudaError_t plan_u13_c64(const PlanItem*, int, const PlanMat*, PlanCtrl*, int, cudaStream_t, int);
cudaError_t plan_herm_u12_c128(const PlanItem*, int, const PlanMat*, PlanCtrl*, int, cudaStream_t, int);
cudaError_t plan_herm_u12_c64(const PlanItem*, int, const PlanMat*, PlanCtrl*, int, cudaStream_t, int);
cudaError_t plan_herm_u13_c128(const PlanItem*, int, const PlanMat*, PlanCtrl*, int, cudaStream_t, int);
cudaError_t plan_herm_u13_c64(const PlanItem*, int, const PlanMat*, PlanCtrl*, int, cudaStream_t, int);

cudaError_t launch_plan(const PlanItem* items, int n_items, const PlanMat* mats, PlanCtrl* ctrl, bool c64, int UB,
                        int blocks_per_sm, cudaStream_t s, int batch, bool herm) {
  if (herm) {
    if (UB == 12)
      return c64 ? plan_herm_u12_c64(items, n_items, mats, ctrl, blocks_per_sm, s, batch)
                 : plan_herm_u12_c128(items, n_items, mats, ctrl, blocks_per_sm, s, batch);
    return c64 ? plan_herm_u13_c64(items, n_items, mats, ctrl, blocks_per_sm, s, batch)
               : plan_herm_u13_c128(items, n_items, mats, ctrl, blocks_per_sm, s, batch);
  }
  if (UB == 12)
    return c64 ? plan_u12_c64(items, n_items, mats, ctrl, blocks_per_sm, s, batch)
               : plan_u12_c128(items, n_items, mats, ctrl, blocks_per_sm, s, batch);
  return c64 ? plan_u13_c64(items, n_items, mats, ctrl, blocks_per_sm, s, batch)
             : plan_u13_c128(items, n_items, mats, ctrl, blocks_per_sm, s, batch);
}

}  // namespace pauli

// Tensor-core (tcgen05) MLP forward/reverse for the FV_TF32 / FV_BF16 paths.
#include "fv_internal.cuh"

namespace fv {

bool tc_supported(const EvalPlan& pl) { (void)pl; return false; }

int mlp_bwd_tc_blocks(fv_ctx ctx, const EvalPlan& pl) { (void)ctx; (void)pl; return -FV_ERR_UNSUPPORTED; }

int launch_mlp_fwd_tc(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xm, const double* Xe,
                      void* U) {
  (void)ctx; (void)pl; (void)params; (void)Xm; (void)Xe; (void)U;
  set_error("tensor-core MLP path not available");
  return FV_ERR_UNSUPPORTED;
}

int launch_mlp_bwd_tc(fv_ctx ctx, const EvalPlan& pl, const void* params, const double* Xm, const double* Xe,
                      const void* UB, double* gpart, int* nb) {
  (void)ctx; (void)pl; (void)params; (void)Xm; (void)Xe; (void)UB; (void)gpart; (void)nb;
  set_error("tensor-core MLP path not available");
  return FV_ERR_UNSUPPORTED;
}

}  // namespace fv

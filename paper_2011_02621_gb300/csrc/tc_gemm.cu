// placeholder: tensor-core steps are not built yet
#include "tn_internal.h"
bool tc_step_supported(const StepParams &) { return false; }
cudaError_t launch_step_tc(int, const StepParams &, const ContractArgs &, const float2 *, const float2 *,
                           const float2 *, float2 *, int *, cudaStream_t) {
  return cudaErrorNotSupported;
}

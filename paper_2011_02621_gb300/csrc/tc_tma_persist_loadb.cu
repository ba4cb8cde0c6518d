// Persistent TMA-fed tcgen05 step: the launches whose overlap operand is loaded as bf16 pieces by
// TMA (the kernel itself is in tc_persist_kernel.cuh).
#include "tc_persist_kernel.cuh"

cudaError_t launch_step_tma_persistent_loadb(const StepParams &s, const ContractArgs &a, const Pieces &A,
                                             const Pieces &B, const OutDesc &out, int *err, cudaStream_t st, int bn,
                                             int64_t c_items, const float2 *ain) {
  return persist_dispatch<0>(s, a, A, B, out, err, st, bn, nullptr, 0, c_items, ain);
}

// Persistent TMA-fed tcgen05 step: the launches whose overlap operand is split from complex64 on
// chip (the kernel itself is in tc_persist_kernel.cuh), and the entry point of both modes.
#include "tc_persist_kernel.cuh"

cudaError_t launch_step_tma_persistent(const StepParams &s, const ContractArgs &a, const Pieces &A, const Pieces &B,
                                       const OutDesc &out, int *err, cudaStream_t st, int bn, const float2 *cbuf,
                                       int64_t c_stride, int64_t c_items, const float2 *ain) {
  if (!cbuf) return launch_step_tma_persistent_loadb(s, a, A, B, out, err, st, bn, c_items, ain);
  return persist_dispatch<2>(s, a, A, B, out, err, st, bn, cbuf, c_stride, c_items, ain);
}

// Persistent form of the TMA-fed tcgen05 step (BF16x6): one CTA per SM walks the output tiles,
// the operand ring runs across tile boundaries and the accumulators are handed between the MMA
// issuer and the epilogue by mbarriers (two TMEM accumulator sets at 64-column tiles).
#pragma once

#include "tn_internal.h"

// Same contract as launch_step_tma for the loaded-B (cbuf == nullptr: B pieces by TMA) and
// complex64-B (cbuf: the overlap tensor [N][K], c_stride elements apart, item i reading copy
// i % c_items, c_items 0 meaning one copy per item) modes. At
// 128-column tiles and K > 64 it issues the same MMAs and sums the accumulators in the same order
// as launch_step_tma (R = 3); at 128-column tiles and K <= 64 it keeps one order-0 accumulator
// (R = 1) and two accumulator sets; at 64-column tiles it uses R = 3 (launch_step_tma: 7). bn: 128 or
// 64 real output columns per tile (0 picks by shape). Returns cudaErrorInvalidValue for
// unsupported shapes or arguments. ain (with cbuf): the step's input as complex64 (item stride
// a.t_stride, row-major [M][K]) instead of the A pieces; the kernel splits it on chip.
cudaError_t launch_step_tma_persistent(const StepParams &s, const ContractArgs &a, const Pieces &A, const Pieces &B,
                                       const OutDesc &out, int *err, cudaStream_t st, int bn, const float2 *cbuf,
                                       int64_t c_stride, int64_t c_items = 0, const float2 *ain = nullptr);

// The loaded-B mode alone (B pieces formed in HBM, c_items copies): launch_step_tma_persistent
// with cbuf == nullptr.
cudaError_t launch_step_tma_persistent_loadb(const StepParams &s, const ContractArgs &a, const Pieces &A,
                                             const Pieces &B, const OutDesc &out, int *err, cudaStream_t st, int bn,
                                             int64_t c_items, const float2 *ain);

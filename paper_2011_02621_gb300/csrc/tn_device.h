// Device helpers shared by the contraction kernels: output stores in the two intermediate
// formats (complex64, or three bf16 pieces per real for a tensor-core consumer).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tn_internal.h"

__device__ __forceinline__ float tn_bf16_round(float x) {   // nearest bf16, as a float
  uint32_t r;
  asm("{\n\t.reg .b16 h;\n\tcvt.rn.bf16.f32 h, %1;\n\tmov.b32 %0, {0, h};\n\t}" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// x = x_0 + x_1 + x_2 with each x_q a bf16 value (the remainders are exact in fp32);
// w[q] packs (re_q, im_q) as a bf16 pair, re in the low half
__device__ __forceinline__ void tn_split3(float x, float y, uint32_t w[3]) {
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float hx = tn_bf16_round(x), hy = tn_bf16_round(y);
    w[q] = (__float_as_uint(hx) >> 16) | (__float_as_uint(hy) & 0xFFFF0000u);
    x -= hx;
    y -= hy;
  }
}

__device__ __forceinline__ void store_out(const OutDesc &o, int64_t t_stride, int64_t item, int64_t off, float2 v) {
  if (o.fmt == 0) {
    reinterpret_cast<float2 *>(o.p)[item * t_stride + off] = v;
  } else {
    uint32_t w[3];
    tn_split3(v.x, v.y, w);
    uint32_t *b = reinterpret_cast<uint32_t *>(o.p) + item * t_stride + off;
    b[0] = w[0];
    b[o.plane_u32] = w[1];
    b[2 * o.plane_u32] = w[2];
  }
}

__device__ __forceinline__ void store_out(const OutDesc &o, int64_t t_stride, int64_t item, int64_t off, double2 v) {
  reinterpret_cast<double2 *>(o.p)[item * t_stride + off] = v;
}

// Device helpers shared by the contraction kernels: output stores in the two intermediate
// formats (complex64, or three bf16 pieces per real for a tensor-core consumer).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tn_internal.h"
#include "tn_smem.h"

// x = x_0 + x_1 + x_2 and y = y_0 + y_1 + y_2 with each piece a bf16 value (nearest, ties to
// even; the remainders are exact in fp32); w[q] packs (x_q, y_q) as a bf16 pair, x in the low
// half, both rounded by one instruction
__device__ __forceinline__ void tn_split3(float x, float y, uint32_t w[3]) {
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    uint32_t h;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(y), "f"(x));
    w[q] = h;
    if (q < 2) {
      x -= __uint_as_float(h << 16);
      y -= __uint_as_float(h & 0xFFFF0000u);
    }
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

// Eight consecutive complex outputs (v[0..15] = re, im pairs) at offsets off .. off + 7 of one
// item: 16-byte vector stores when off is aligned for them, scalar stores otherwise.
__device__ __forceinline__ void store_out8(const OutDesc &o, int64_t t_stride, int64_t item, int64_t off,
                                           const float v[16]) {
  if (o.fmt == 0) {
    float2 *b = reinterpret_cast<float2 *>(o.p) + item * t_stride + off;
    if ((off & 1) == 0) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        reinterpret_cast<float4 *>(b)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = make_float2(v[2 * j], v[2 * j + 1]);
    }
  } else {
    uint32_t w[3][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint32_t t[3];
      tn_split3(v[2 * j], v[2 * j + 1], t);
      w[0][j] = t[0];
      w[1][j] = t[1];
      w[2][j] = t[2];
    }
    uint32_t *b = reinterpret_cast<uint32_t *>(o.p) + item * t_stride + off;
    if ((off & 3) == 0) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        uint4 *d = reinterpret_cast<uint4 *>(b + q * o.plane_u32);
        d[0] = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
        d[1] = make_uint4(w[q][4], w[q][5], w[q][6], w[q][7]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int j = 0; j < 8; ++j) b[q * o.plane_u32 + j] = w[q][j];
    }
  }
}

// Four consecutive complex outputs (v[0..7]) at offsets off .. off + 3 of one item.
__device__ __forceinline__ void store_out4(const OutDesc &o, int64_t t_stride, int64_t item, int64_t off,
                                           const float v[8]) {
  if (o.fmt == 0) {
    float2 *b = reinterpret_cast<float2 *>(o.p) + item * t_stride + off;
    if ((off & 1) == 0) {
      reinterpret_cast<float4 *>(b)[0] = make_float4(v[0], v[1], v[2], v[3]);
      reinterpret_cast<float4 *>(b)[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = make_float2(v[2 * j], v[2 * j + 1]);
    }
  } else {
    uint32_t w[3][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t t[3];
      tn_split3(v[2 * j], v[2 * j + 1], t);
      w[0][j] = t[0];
      w[1][j] = t[1];
      w[2][j] = t[2];
    }
    uint32_t *b = reinterpret_cast<uint32_t *>(o.p) + item * t_stride + off;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if ((off & 3) == 0) {
        *reinterpret_cast<uint4 *>(b + q * o.plane_u32) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) b[q * o.plane_u32 + j] = w[q][j];
      }
    }
  }
}

__device__ __forceinline__ void store_out4(const OutDesc &o, int64_t t_stride, int64_t item, int64_t off,
                                           const double v[8]) {
  double2 *b = reinterpret_cast<double2 *>(o.p) + item * t_stride + off;
#pragma unroll
  for (int j = 0; j < 4; ++j) b[j] = make_double2(v[2 * j], v[2 * j + 1]);
}

// columns n .. n + len - 1 of a step land on consecutive output offsets, in order
__device__ __forceinline__ bool tn_contig(const int32_t *ocol, int64_t n, int len) {
  const int32_t o = ocol[n];
  bool ok = true;
#pragma unroll
  for (int i = 1; i < len; ++i) ok = ok && ocol[n + i] == o + i;
  return ok;
}

// The 16 fp32 results v (eight complex columns n0 .. n0 + 7 of one row, ro its row offset) of a
// tensor-core epilogue into the next step's layout: one eight-wide store when the eight columns
// are consecutive there, else four-wide stores for consecutive groups of four, else one by one.
__device__ __forceinline__ void store_cols8(const OutDesc &o, int64_t t_stride, int64_t item, int64_t ro,
                                            const int32_t *ocol, int64_t n0, int64_t N, const float v[16]) {
  if (n0 + 7 < N && tn_contig(ocol, n0, 8)) {
    store_out8(o, t_stride, item, ro + ocol[n0], v);
    return;
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t nb = n0 + 4 * h;
    if (nb + 3 < N && tn_contig(ocol, nb, 4)) {
      store_out4(o, t_stride, item, ro + ocol[nb], v + 8 * h);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (nb + j < N) store_out(o, t_stride, item, ro + ocol[nb + j], make_float2(v[8 * h + 2 * j], v[8 * h + 2 * j + 1]));
    }
  }
}

// ---- overlap elements and item context (shared by the formation, SIMT and TMA kernels)

template <typename V> __device__ __forceinline__ V cz() { V v; v.x = 0; v.y = 0; return v; }
template <typename V> __device__ __forceinline__ V cfma(V a, V b, V c) {
  c.x = fma(a.x, b.x, fma(-a.y, b.y, c.x));
  c.y = fma(a.x, b.y, fma(a.y, b.x, c.y));
  return c;
}

struct ItemCtx {
  int64_t b, sl;
  int32_t sa, sb;
};

__device__ __forceinline__ ItemCtx item_ctx(const ContractArgs &a, const StepParams &s, int64_t item) {
  ItemCtx c;
  if (a.n_slices == 1) {
    c.b = item;
    c.sl = a.slice0;
  } else {
    c.b = (unsigned)item / (unsigned)a.n_slices;
    c.sl = a.slice0 + (unsigned)item % (unsigned)a.n_slices;
  }
  c.sa = a.tab[s.t_sa + c.sl];
  c.sb = a.tab[s.t_sb + c.sl];
  return c;
}

// output offset of row m: m decomposed over the rest legs, weighted by their output strides
__device__ __forceinline__ int orow_of(const StepParams &s, int64_t m64) {
  unsigned m = (unsigned)m64;   // rows < 2^31 (checked when the plan is compiled)
  int off = 0;
  if (s.rest_pow2) {
    for (int j = s.n_rest - 1; j >= 0; --j) {
      const int lg = s.rest_log2[j];
      off += (int)(m & ((1u << lg) - 1u)) * s.rest_ostride[j];
      m >>= lg;
    }
  } else {
    for (int j = s.n_rest - 1; j >= 0; --j) {
      const unsigned d = (unsigned)s.rest_dim[j];
      off += (int)(m % d) * s.rest_ostride[j];
      m /= d;
    }
  }
  return off;
}

// C element (Eq. overlap) at table offsets: the sum over the node's physical index (two values,
// or 4 / 8 for a node that absorbed neighbours), in index order
template <typename V>
__device__ __forceinline__ V overlap_elem(const V *ket, const V *bra, int64_t ia, int64_t ib, int64_t ksig,
                                          int64_t bsig, int64_t phys) {
  V acc = cfma(ket[ia + ksig], bra[ib + bsig], cfma(ket[ia], bra[ib], cz<V>()));
  for (int64_t q = 2; q < phys; ++q) acc = cfma(ket[ia + q * ksig], bra[ib + q * bsig], acc);
  return acc;
}

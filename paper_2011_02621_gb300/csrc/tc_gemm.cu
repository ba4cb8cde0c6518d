// Tensor-core (tcgen05) contraction step for complex64 intermediates.
//
// One absorption step is the complex GEMM  T_out[orow(m) + ocol[n]] = sum_k T_in[m*K + k] * C[k][n]
// with C the overlap tensor of the absorbed node (Eq. overlap), formed beforehand per item as
// [N][K] by the overlap-formation kernel, and the output written straight into the layout of
// the next step (the transposes of transpose-transpose-GEMM live in this store). It runs as
// one real GEMM on the 5th-generation tensor cores: the complex64 A rows are read as
// interleaved (re, im) floats (K_r = 2K), and B is the real embedding of C,
//     B_r[2k][2n] = Re c, B_r[2k][2n+1] = Im c, B_r[2k+1][2n] = -Im c, B_r[2k+1][2n+1] = Re c,
// so the fp32 accumulator D[m][2n + {0,1}] is (Re, Im) of the complex result.
//
// Each CTA (4 warps) owns one 128 x BN real output tile of one item. All warps load the A
// rows and the C rows with coalesced loads and write the tiles (B in its real embedding), split into
// P pieces of the operand type (x = x_0 + x_1 + ..., each piece exactly representable),
// directly in 128-byte-swizzled K-major shared memory; thread 0 issues tcgen05.mma
// (kind::tf32 or kind::f16 with bf16 operands, FP32 accumulators in TMEM) for every product
// x_i * y_j with i + j <= ORD -- one accumulator per order i + j, so that the small
// correction terms keep their low bits -- and commits each stage to an mbarrier. Two stages
// alternate; every wait is bounded by a clock limit and reports an error code instead of
// hanging. The epilogue reads the accumulators with tcgen05.ld and sums them, smallest first.
//
// Forms: TF32 (P=1), TF32x3 (P=2, 3 products), BF16x3 (P=2), BF16x6 (P=3, 6 products, about
// 24 significant bits per product), TF32x6 (P=3, 6 products).
#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_ptx.h"
#include "tn_device.h"
#include "tn_internal.h"

namespace {

constexpr int TC_THREADS = 256;   // 8 warps: all load and split operands, warp 0 lane 0 issues MMAs
constexpr int BM = 128;          // rows per tile (M of the MMA)
constexpr long long WAIT_CYCLES = 500000000LL;    // ~0.25 s at 2 GHz

using tcx::s_u32;

// 128B swizzle (Swizzle<3,4,3>): XOR the 16-byte chunk index with the row within the 8-row atom
__device__ __forceinline__ uint32_t swz(uint32_t off) { return off ^ (((off >> 7) & 7u) << 4); }

// bounded wait: false (and an error code) if the phase did not complete within the limit
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int *err, int code) {
  return tcx::bar_wait(a, parity, err, code, WAIT_CYCLES);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ float bf16_rn(float x) {   // round to the nearest bf16, returned as a float
  uint32_t r;
  asm("{\n\t.reg .b16 h;\n\tcvt.rn.bf16.f32 h, %1;\n\tmov.b32 %0, {0, h};\n\t}" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Operand kinds: tf32 (4-byte elements, MMA K = 8) or bf16 (2-byte elements, MMA K = 16).
// A stage row is always 128 bytes (one 128B swizzle row), i.e. BKR = 32 tf32 or 64 bf16 reals.
template <int KIND> struct Op;
template <> struct Op<0> {
  static constexpr int ELEM = 4;
  static __device__ __forceinline__ float round(float x) { return tf32_rna(x); }
  static __device__ __forceinline__ void st(uint8_t *tile, int row, int kr, float x, float y) {
    *reinterpret_cast<float2 *>(tile + swz((uint32_t)(row * 128 + kr * 4))) = make_float2(x, y);
  }
  static __device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
  }
  static constexpr uint32_t FMT = 2;   // tf32
};
template <> struct Op<1> {
  static constexpr int ELEM = 2;
  static __device__ __forceinline__ float round(float x) { return bf16_rn(x); }
  static __device__ __forceinline__ void st(uint8_t *tile, int row, int kr, float x, float y) {
    // x, y are exact bf16 values: keep their upper halves
    const uint32_t w = (__float_as_uint(x) >> 16) | (__float_as_uint(y) & 0xFFFF0000u);
    *reinterpret_cast<uint32_t *>(tile + swz((uint32_t)(row * 128 + kr * 2))) = w;
  }
  static __device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
  }
  static constexpr uint32_t FMT = 1;   // bf16
};

template <int KIND>
__device__ __forceinline__ uint32_t make_idesc_k(int bn) {
  uint32_t d = 0;
  d |= 1u << 4;                          // D format f32
  d |= Op<KIND>::FMT << 7;               // A format
  d |= Op<KIND>::FMT << 10;              // B format
  d |= (uint32_t)(bn >> 3) << 17;        // N / 8
  d |= (uint32_t)(BM >> 4) << 24;        // M / 16
  return d;
}

// store a (K, K+1) pair split into P pieces of the operand kind: x = x_0 + x_1 + ... (each exact)
template <int KIND, int P>
__device__ __forceinline__ void st_pieces(uint8_t *base, int piece_bytes, int row, int kr, float x, float y) {
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const float hx = Op<KIND>::round(x), hy = Op<KIND>::round(y);
    Op<KIND>::st(base + q * piece_bytes, row, kr, hx, hy);
    x -= hx;
    y -= hy;
  }
}

__host__ __device__ constexpr int next_pow2(int x) { return x <= 32 ? 32 : x <= 64 ? 64 : x <= 128 ? 128 : x <= 256 ? 256 : 512; }

// KIND: 0 tf32, 1 bf16. P: pieces per operand. ORD: keep products x_i * y_j with i + j <= ORD,
// accumulated per order i + j in separate TMEM accumulators and summed (small first) at the end.
// R: the order-0 products (the large ones) are spread round-robin over R accumulators by MMA
// k-step, so that each accumulator sums 1/R of the k-steps: the tensor core aligns and truncates
// when it accumulates, and the error of that grows with the number of accumulations.
template <int KIND, int P, int ORD, int BN, int R>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_step_kernel(StepParams s, ContractArgs a, const float2 *__restrict__ cbuf, int64_t c_stride,
               const float2 *__restrict__ tin, float2 *__restrict__ tout, int *err) {
  constexpr int ELEM = Op<KIND>::ELEM;
  constexpr int BKR = 128 / ELEM;                // real K per stage (one 128-byte swizzle row)
  constexpr int BKC = BKR / 2;                   // complex K per stage
  constexpr int A_BYTES = BM * 128;              // one piece of the A tile
  constexpr int B_BYTES = BN * 128;              // one piece of the B tile
  constexpr int STAGE = P * (A_BYTES + B_BYTES); // A pieces, then B pieces
  constexpr int GROUPS = ORD + R;                // accumulators: R for order 0, one per order >= 1
  constexpr uint32_t TMEM_COLS = (uint32_t)next_pow2(GROUPS * BN);
  constexpr int KSTEPS = 128 / 32;               // 32 bytes of K per MMA instruction
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ int rowoff[BM];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t tiles_m = (s.M + BM - 1) / BM, tiles_n = (2 * s.N + BN - 1) / BN;
  const int64_t blk = blockIdx.x;
  const int64_t item = blk / (tiles_m * tiles_n);
  const int64_t rem = blk % (tiles_m * tiles_n);
  const int64_t m0 = (rem / tiles_n) * BM;
  const int64_t nr0 = (rem % tiles_n) * BN;      // first real output column
  const float2 *tp = tin + item * a.t_stride;
  const float2 *cp = cbuf + item * c_stride;
  const int32_t *ocol = a.tab + s.t_ocol;

  if (tid == 0) {
    tcx::bar_init(s_u32(&mbar[0]), 1);
    tcx::bar_init(s_u32(&mbar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(&tmem_base_s)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid < BM) {
    const int64_t m = m0 + tid;
    int off = -1;
    if (m < s.M) {
      off = 0;
      unsigned r = (unsigned)m;
      for (int j = s.n_rest - 1; j >= 0; --j) {
        if (s.rest_pow2) {
          off += (int)(r & ((1u << s.rest_log2[j]) - 1u)) * s.rest_ostride[j];
          r >>= s.rest_log2[j];
        } else {
          const unsigned d = (unsigned)s.rest_dim[j];
          off += (int)(r % d) * s.rest_ostride[j];
          r /= d;
        }
      }
    }
    rowoff[tid] = off;                           // output row offset in the next layout
  }
  tcx::fence_before();
  __syncthreads();
  tcx::fence_after();
  const uint32_t tmem = tmem_base_s;
  const uint32_t idesc = make_idesc_k<KIND>(BN);
  const int64_t nk = (s.K + BKC - 1) / BKC;
  bool bad = false;

  // operand values of one chunk per thread, loaded ahead of their shared-memory stores
  constexpr int NA = BM * BKC / TC_THREADS, NB = (BN / 2) * BKC / TC_THREADS;
  static_assert(NA * TC_THREADS == BM * BKC && NB * TC_THREADS == (BN / 2) * BKC, "tile split");
  float2 va[NA], vb[NB];
  auto load_chunk = [&](int64_t kc) {
    const int64_t k0 = kc * BKC;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const int e = tid + TC_THREADS * i, row = e / BKC, kk = e % BKC;
      const int64_t m = m0 + row, k = k0 + kk;
      va[i] = (m < s.M && k < s.K) ? tp[m * s.K + k] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int e = tid + TC_THREADS * i, nl = e / BKC, kk = e % BKC;
      const int64_t n = nr0 / 2 + nl, k = k0 + kk;
      vb[i] = (n < s.N && k < s.K) ? cp[n * s.K + k] : make_float2(0.f, 0.f);
    }
  };
  if (nk > 0) load_chunk(0);
  int64_t issued = 0;
  for (int64_t kc = 0; kc < nk; ++kc) {
    const int st = (int)(kc & 1);
    uint8_t *Ab = smem + st * STAGE, *Bb = Ab + P * A_BYTES;
    if (kc >= 2 && !bad) {
      // the MMAs that last read this stage (chunk kc-2) must be complete before it is overwritten
      if (!mbar_wait(s_u32(&mbar[st]), (uint32_t)(((kc - 2) >> 1) & 1), err, 1)) bad = true;
    }
    if (__syncthreads_or(bad)) { bad = true; break; }
    // ---- A tile (rows of T_in) and B tile (real embedding of C: row 2n (Re, -Im), row 2n+1 (Im, Re))
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const int e = tid + TC_THREADS * i;
      st_pieces<KIND, P>(Ab, A_BYTES, e / BKC, 2 * (e % BKC), va[i].x, va[i].y);
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int e = tid + TC_THREADS * i, nl = e / BKC, kk = e % BKC;
      st_pieces<KIND, P>(Bb, B_BYTES, 2 * nl, 2 * kk, vb[i].x, -vb[i].y);
      st_pieces<KIND, P>(Bb, B_BYTES, 2 * nl + 1, 2 * kk, vb[i].y, vb[i].x);
    }
    if (kc + 1 < nk) load_chunk(kc + 1);         // next chunk's loads overlap this chunk's MMAs
    tcx::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tcx::fence_after();
      const uint32_t a0 = s_u32(Ab), b0 = s_u32(Bb);
#pragma unroll
      for (int ks = 0; ks < KSTEPS; ++ks) {
        const uint32_t off = (uint32_t)ks * 32u;
        const int64_t t = kc * KSTEPS + ks;           // global k-step
        const bool first = (t == 0);
        // order 0 -> accumulator t % R (first use: t < R); order o >= 1 -> accumulator R + o - 1
        Op<KIND>::mma(tmem + (uint32_t)((t % R) * BN), tcx::desc_sw128(a0 + off), tcx::desc_sw128(b0 + off), idesc,
                      t < R ? 0u : 1u);
#pragma unroll
        for (int o = 1; o <= ORD; ++o) {
#pragma unroll
          for (int i = 0; i < P; ++i) {
            const int j = o - i;
            if (j < 0 || j >= P) continue;
            const uint32_t acc = (first && i == (o < P ? 0 : o - P + 1)) ? 0u : 1u;
            Op<KIND>::mma(tmem + (uint32_t)((R + o - 1) * BN), tcx::desc_sw128(a0 + i * A_BYTES + off),
                          tcx::desc_sw128(b0 + j * B_BYTES + off), idesc, acc);
          }
        }
      }
      tcx::mma_commit_to(s_u32(&mbar[st]));
    }
    ++issued;
  }
  // ---- wait for the last committed stage (commits complete in order); also after an error,
  // so that no MMA is still reading shared memory or writing TMEM when the CTA frees them
  if (issued > 0) {
    const int64_t last = issued - 1;
    if (!mbar_wait(s_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1), err, 2)) bad = true;
  }
  bad = __syncthreads_or(bad);
  tcx::fence_after();
  if (!bad && issued == nk) {
    // ---- epilogue: warp w reads TMEM lanes 32(w%4).. (rows) and half (w/4) of the columns, 16 at a
    // time, and adds the accumulators from the smallest up
    const int lg = warp & 3, half = warp >> 2;
    const int ro = rowoff[lg * 32 + lane];
    float2 *op = tout + item * a.t_stride;
#pragma unroll 1
    for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 16) {
      float acc[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = 0.f;
#pragma unroll
      for (int g = GROUPS - 1; g >= 0; --g) {
        if (g < R && (int64_t)g >= nk * KSTEPS) continue;   // order-0 accumulator never written
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(g * BN + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] += __uint_as_float(r[j]);
      }
      if (ro >= 0) {
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const int64_t n = (nr0 + c0 + j) >> 1;
          if (n < s.N) op[ro + ocol[n]] = make_float2(acc[j], acc[j + 1]);
        }
      }
    }
  }
  tcx::fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

template <int KIND, int P, int ORD, int BN, int R>
cudaError_t launch_bn(const StepParams &s, const ContractArgs &a, const float2 *cbuf, int64_t c_stride,
                      const float2 *tin, float2 *tout, int *err, cudaStream_t st) {
  constexpr size_t stage = (size_t)P * (BM * 128 + BN * 128);
  const size_t smem = 2 * stage + 1024;
  static_assert(2 * (size_t)P * (BM * 128 + BN * 128) + 1024 <= 227 * 1024, "shared memory");
  // the dynamic shared memory limit on the current device (set once per device)
  const int lim = tn_smem_optin<tc_step_kernel<KIND, P, ORD, BN, R>>();
  if (lim < 0 || (size_t)lim < smem) return cudaErrorInvalidValue;
  const int64_t tiles = ((s.M + BM - 1) / BM) * ((2 * s.N + BN - 1) / BN);
  const int64_t grid = tiles * a.items;
  if (grid <= 0) return cudaSuccess;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  tc_step_kernel<KIND, P, ORD, BN, R><<<(unsigned)grid, TC_THREADS, smem, st>>>(s, a, cbuf, c_stride, tin, tout, err);
  tn_count_launch(1);
  return cudaGetLastError();
}

// tile width and accumulator split: (R + ORD) * BN <= 512 TMEM columns
template <int KIND, int P, int ORD>
cudaError_t launch_form_p(const StepParams &s, const ContractArgs &a, const float2 *cbuf, int64_t c_stride,
                          const float2 *tin, float2 *tout, int *err, cudaStream_t st) {
  const int64_t nr = 2 * s.N;
  if constexpr (ORD == 0) {
    if (nr >= 256) return launch_bn<KIND, P, ORD, 256, 2>(s, a, cbuf, c_stride, tin, tout, err, st);
    if (nr >= 128) return launch_bn<KIND, P, ORD, 128, 4>(s, a, cbuf, c_stride, tin, tout, err, st);
    return launch_bn<KIND, P, ORD, 64, 8>(s, a, cbuf, c_stride, tin, tout, err, st);
  } else {
    if (nr >= 128) return launch_bn<KIND, P, ORD, 128, 4 - ORD>(s, a, cbuf, c_stride, tin, tout, err, st);
    return launch_bn<KIND, P, ORD, 64, 8 - ORD>(s, a, cbuf, c_stride, tin, tout, err, st);
  }
}

}  // namespace

bool tc_step_supported(const StepParams &s) {
  // a 128-row tile must be mostly useful; small outputs stay on the SIMT kernels
  return s.M >= 64 && 2 * s.N >= 32 && s.K >= 8;
}

cudaError_t launch_step_tc(int prec, const StepParams &s, const ContractArgs &a, const float2 *cbuf, int64_t c_stride,
                           const float2 *tin, float2 *tout, int *err, cudaStream_t st) {
  switch (prec) {
    case TN_TF32: return launch_form_p<0, 1, 0>(s, a, cbuf, c_stride, tin, tout, err, st);
    case TN_TF32X3: return launch_form_p<0, 2, 1>(s, a, cbuf, c_stride, tin, tout, err, st);
    case TN_BF16X3: return launch_form_p<1, 2, 1>(s, a, cbuf, c_stride, tin, tout, err, st);
    case TN_BF16X6: return launch_form_p<1, 3, 2>(s, a, cbuf, c_stride, tin, tout, err, st);
    case TN_TF32X6: return launch_form_p<0, 3, 2>(s, a, cbuf, c_stride, tin, tout, err, st);
    default: return cudaErrorNotSupported;
  }
}

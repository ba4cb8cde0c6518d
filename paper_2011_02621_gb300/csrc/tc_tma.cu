// TMA-fed tcgen05 contraction step (BF16x6 form): the operand path uses no CUDA-core work.
//
// Operands arrive pre-split. Every complex64 value x of an intermediate that feeds a
// tensor-core step is stored by its producer as three bf16 planes x = x_0 + x_1 + x_2 (each
// piece exact), in the consumer's row-major [M][2K] layout (interleaved re, im). The overlap
// tensor C of the absorbed node (Eq. overlap) is written by the formation kernel in its real
// embedding B_r[2N][2K] (row 2n = (Re c, -Im c), row 2n+1 = (Im c, Re c) along k), split the
// same way. One CTA computes a 128 x BN real output tile of one item:
//   warp 0   issues cp.async.bulk.tensor loads of the 3 A and 3 B pieces of each 64-real K
//            chunk into a ring of shared-memory stages (128-byte swizzle, the canonical
//            K-major layout of the MMA), signalling a "full" mbarrier with the byte count;
//   warp 1   allocates TMEM and issues tcgen05.mma kind::f16 (bf16 in, fp32 accumulate) for
//            the six products x_i*y_j with i + j <= 2, order 0 spread round-robin over R
//            accumulators, orders 1 and 2 together in one more; each stage is released by
//            tcgen05.commit on its "empty" mbarrier, the last one on "done";
//   warps 2-5 wait for "done", read the accumulators with tcgen05.ld, add them smallest first
//            and write the result straight into the next step's layout, as complex64 or as
//            bf16 pieces for the next tensor-core step.
// B modes. BM 0: the B pieces are loaded by TMA (formed beforehand). BM 1: no overlap tensor is
// stored at all: during the main loop warps 2-5 compute each stage's B tile themselves from the
// absorbed node's ket and bra tensors (Eq. overlap, the same arithmetic as the formation
// kernel). BM 2: warps 2-5 read the overlap tensor as complex64 [N][K] (8 bytes per element,
// independent coalesced loads, all of a stage's loads issued before any is used). In modes 1 and
// 2 the warps split the tile into the three bf16 pieces and store it in the 128-byte-swizzled
// K-major layout the MMA reads; each of those 128 threads then makes its writes visible to the
// tensor core's async proxy and arrives on the stage's "full" mbarrier next to the TMA's byte
// count. Only the A pieces come through TMA.
// Every wait is bounded by a clock limit and raises an error code instead of hanging.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tc_ptx.h"
#include "tn_device.h"
#include "tn_internal.h"

namespace {

constexpr int T_THREADS = 192;
constexpr int T_BM = 128;
constexpr int T_P = 3;
constexpr long long T_WAIT = 500000000LL;   // ~0.25 s at 2 GHz

using tcx::bar_arrive;
using tcx::bar_expect_tx;
using tcx::bar_init;
using tcx::desc_sw128;
using tcx::mma_bf16;
using tcx::mma_commit_to;
using tcx::s_u32;
using tcx::sts128;
using tcx::sw128_off;
using tcx::tma_3d;

__device__ __forceinline__ uint32_t idesc_bf16(int bn) { return tcx::idesc_bf16(T_BM, bn); }

// bounded wait: after T_WAIT clocks the error code is recorded and the wait gives up
__device__ __forceinline__ bool bar_wait(uint32_t a, uint32_t parity, int *err, int code) {
  return tcx::bar_wait(a, parity, err, code, T_WAIT);
}

}  // namespace

namespace {

template <int BN, int R, int S, int BM>
__global__ void __launch_bounds__(T_THREADS, 1)
tma_step_kernel(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
                const __grid_constant__ CUtensorMap tA2, const __grid_constant__ CUtensorMap tB0,
                const __grid_constant__ CUtensorMap tB1, const __grid_constant__ CUtensorMap tB2, StepParams s,
                ContractArgs a, OutDesc out, int *err, const float2 *ket, const float2 *bra, const float2 *cbuf,
                int64_t c_stride, int64_t c_items, int staged) {
  constexpr bool BUILD = BM != 0;
  constexpr int A_BYTES = T_BM * 128, B_BYTES = BN * 128;
  constexpr int STAGE = T_P * (A_BYTES + B_BYTES);
  constexpr int GROUPS = R + 1;                  // R order-0 accumulators + one for orders 1 and 2
  constexpr uint32_t TMEM_COLS = GROUPS * BN <= 32 ? 32 : GROUPS * BN <= 64 ? 64 : GROUPS * BN <= 128 ? 128
                                 : GROUPS * BN <= 256 ? 256 : 512;
  static_assert(GROUPS * BN <= 512, "TMEM columns");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[S], empty[S], done;
  __shared__ uint32_t tmem_s;
  __shared__ int rowoff[T_BM];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t tiles_m = (s.M + T_BM - 1) / T_BM, tiles_n = (2 * s.N + BN - 1) / BN;
  const int64_t blk = blockIdx.x;
  const int item = (int)(blk / (tiles_m * tiles_n));
  const int64_t rem = blk % (tiles_m * tiles_n);
  const int m0 = (int)((rem / tiles_n) * T_BM);
  const int nr0 = (int)((rem % tiles_n) * BN);
  const int64_t nk = (2 * s.K + 63) / 64;        // 64-real K chunks

  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      bar_init(s_u32(&full[i]), BUILD ? 1 + 4 * 32 : 1);   // TMA (+ the 128 B builders)
      bar_init(s_u32(&empty[i]), 1);
    }
    bar_init(s_u32(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(&tmem_s)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid >= 64 && tid < 64 + T_BM) {            // epilogue warps: output row offsets
    const int r = tid - 64;
    const int64_t m = m0 + r;
    int off = -1;
    if (m < s.M) {
      off = 0;
      unsigned mm = (unsigned)m;
      for (int j = s.n_rest - 1; j >= 0; --j) {
        if (s.rest_pow2) {
          off += (int)(mm & ((1u << s.rest_log2[j]) - 1u)) * s.rest_ostride[j];
          mm >>= s.rest_log2[j];
        } else {
          const unsigned d = (unsigned)s.rest_dim[j];
          off += (int)(mm % d) * s.rest_ostride[j];
          mm /= d;
        }
      }
    }
    rowoff[r] = off;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_s;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      const CUtensorMap *mA[3] = {&tA0, &tA1, &tA2};
      const CUtensorMap *mB[3] = {&tB0, &tB1, &tB2};
      int64_t issued = 0;
      for (int64_t kc = 0; kc < nk; ++kc) {
        const int st = (int)(kc % S);
        const uint32_t it = (uint32_t)(kc / S);
        if (kc >= S && !bar_wait(s_u32(&empty[st]), (it - 1) & 1, err, 11)) break;
        uint8_t *base = smem + st * STAGE;
        bar_expect_tx(s_u32(&full[st]), (uint32_t)(BUILD ? T_P * A_BYTES : STAGE));
        for (int q = 0; q < T_P; ++q)
          tma_3d(s_u32(base + q * A_BYTES), mA[q], (int)(kc * 64), m0, item, s_u32(&full[st]));
        if (!BUILD)
          for (int q = 0; q < T_P; ++q)
            tma_3d(s_u32(base + T_P * A_BYTES + q * B_BYTES), mB[q], (int)(kc * 64), nr0, item, s_u32(&full[st]));
        ++issued;
      }
      if (issued > 0) {   // the last loads must have landed before the CTA may exit
        const int64_t last = issued - 1;
        bar_wait(s_u32(&full[last % S]), (uint32_t)((last / S) & 1), err, 12);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(BN);
      for (int64_t kc = 0; kc < nk; ++kc) {
        const int st = (int)(kc % S);
        if (!bar_wait(s_u32(&full[st]), (uint32_t)((kc / S) & 1), err, 13)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = s_u32(smem + st * STAGE), b0 = a0 + T_P * A_BYTES;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {          // 16 bf16 (32 bytes) of K per instruction
          const uint32_t off = (uint32_t)ks * 32u;
          const int64_t t = kc * 4 + ks;
          const uint32_t first = (t == 0) ? 0u : 1u;
          mma_bf16(tmem + (uint32_t)((t % R) * BN), desc_sw128(a0 + off), desc_sw128(b0 + off), idesc,
                   t < R ? 0u : 1u);
          // orders 1 and 2 in one accumulator: x0*y1 + x1*y0, then x0*y2 + x1*y1 + x2*y0 (order-2
          // terms, ~2^-16 of a product, lie far above that accumulator's truncation level)
          mma_bf16(tmem + (uint32_t)(R * BN), desc_sw128(a0 + off), desc_sw128(b0 + B_BYTES + off), idesc, first);
          mma_bf16(tmem + (uint32_t)(R * BN), desc_sw128(a0 + A_BYTES + off), desc_sw128(b0 + off), idesc, 1u);
          mma_bf16(tmem + (uint32_t)(R * BN), desc_sw128(a0 + off), desc_sw128(b0 + 2 * B_BYTES + off), idesc, 1u);
          mma_bf16(tmem + (uint32_t)(R * BN), desc_sw128(a0 + A_BYTES + off), desc_sw128(b0 + B_BYTES + off), idesc,
                   1u);
          mma_bf16(tmem + (uint32_t)(R * BN), desc_sw128(a0 + 2 * A_BYTES + off), desc_sw128(b0 + off), idesc, 1u);
        }
        mma_commit_to(s_u32(&empty[st]));
      }
      mma_commit_to(s_u32(&done));               // after every issued MMA, also on an early stop
    }
  } else {
    if (BUILD) {
      // ---------------- B builders (warps 2..5): stage kc's B tile, real rows nr0 .. nr0 + BN - 1
      // (complex column n = row / 2; row 2n = (Re c, -Im c), row 2n + 1 = (Im c, Re c) along k),
      // reals kc*64 .. kc*64 + 63 (complex k = kc*32 .. kc*32 + 31); zeros outside K and N
      const int bt = tid - 64;
      const ItemCtx c = item_ctx(a, s, item);
      const float2 *kp = ket + s.ket_off + c.sa;
      const float2 *bp = bra + c.b * a.bra_stride + s.bra_off + c.sb;
      if (BM == 1 && staged) {
        // the node's ket and bra tensors (small) into shared memory past the stage ring, once
        float2 *nodes = reinterpret_cast<float2 *>(smem + S * STAGE);
        const int64_t tk = s.phys * s.ket_sig, tb = s.phys * s.bra_sig;
        const float2 *kg = ket + s.ket_off, *bg = bra + c.b * a.bra_stride + s.bra_off;
        for (int64_t i = bt; i < tk; i += 128) nodes[i] = kg[i];
        for (int64_t i = bt; i < tb; i += 128) nodes[tk + i] = bg[i];
        asm volatile("bar.sync 1, 128;" ::: "memory");   // the four builder warps only
        kp = nodes + c.sa;
        bp = nodes + tk + c.sb;
      }
      const int32_t *bka = a.tab + s.t_bka, *bkb = a.tab + s.t_bkb;
      const int32_t *bna = a.tab + s.t_bna, *bnb = a.tab + s.t_bnb;
      const int64_t n_base = nr0 >> 1;
      if (BM == 2) {
        // software-pipelined: the next stage's loads are issued before this stage waits for its
        // buffer and splits (tasks: four consecutive complex k of one column n)
        constexpr int TASKS = (BN / 2) * 8 / 128;
        float4 xn[TASKS][2];
        auto load = [&](int64_t kc, float4 (&x)[TASKS][2]) {
#pragma unroll
          for (int j = 0; j < TASKS; ++j) {
            const int t = bt + 128 * j, c16 = t & 7, nl = t >> 3;
            const int64_t n = n_base + nl, k0 = kc * 32 + c16 * 4;
            x[j][0] = x[j][1] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (n < s.N && k0 < s.K) {   // K % 4 == 0: the four k are all in range or all out
              const float4 *src = reinterpret_cast<const float4 *>(cbuf + (item % c_items) * c_stride + n * s.K + k0);
              x[j][0] = __ldg(src);
              x[j][1] = __ldg(src + 1);
            }
          }
        };
        if (nk > 0) load(0, xn);
        for (int64_t kc = 0; kc < nk; ++kc) {
          float4 x[TASKS][2];
#pragma unroll
          for (int j = 0; j < TASKS; ++j) {
            x[j][0] = xn[j][0];
            x[j][1] = xn[j][1];
          }
          if (kc + 1 < nk) load(kc + 1, xn);
          const int st = (int)(kc % S);
          const uint32_t it = (uint32_t)(kc / S);
          if (kc >= S && !bar_wait(s_u32(&empty[st]), (it - 1) & 1, err, 15)) break;
          const uint32_t bbase = s_u32(smem + st * STAGE + T_P * A_BYTES);
#pragma unroll
          for (int j = 0; j < TASKS; ++j) {
            const int t = bt + 128 * j, c16 = t & 7, nl = t >> 3;
            const float re[4] = {x[j][0].x, x[j][0].z, x[j][1].x, x[j][1].z};
            const float im[4] = {x[j][0].y, x[j][0].w, x[j][1].y, x[j][1].w};
            uint32_t w0[T_P][4], w1[T_P][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              uint32_t t0[T_P], t1[T_P];
              tn_split3(re[i], -im[i], t0);
              tn_split3(im[i], re[i], t1);
#pragma unroll
              for (int q = 0; q < T_P; ++q) {
                w0[q][i] = t0[q];
                w1[q][i] = t1[q];
              }
            }
#pragma unroll
            for (int q = 0; q < T_P; ++q) {
              sts128(bbase + q * B_BYTES + sw128_off(2 * nl, c16), w0[q]);
              sts128(bbase + q * B_BYTES + sw128_off(2 * nl + 1, c16), w1[q]);
            }
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          bar_arrive(s_u32(&full[st]));
        }
      } else
      for (int64_t kc = 0; kc < nk; ++kc) {
        const int st = (int)(kc % S);
        const uint32_t it = (uint32_t)(kc / S);
        if (kc >= S && !bar_wait(s_u32(&empty[st]), (it - 1) & 1, err, 15)) break;
        const uint32_t bbase = s_u32(smem + st * STAGE + T_P * A_BYTES);
        for (int t = bt; t < (BN / 2) * 8; t += 128) {
          const int c16 = t & 7, nl = t >> 3;        // 16-byte chunk = four complex k; complex column
          const int64_t n = n_base + nl;
          const int64_t k0 = kc * 32 + c16 * 4;
          int64_t ia_n = 0, ib_n = 0;
          if (n < s.N) {
            ia_n = bna[n];
            ib_n = bnb[n];
          }
          uint32_t w0[T_P][4], w1[T_P][4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int64_t k = k0 + i;
            float2 v = make_float2(0.f, 0.f);
            if (n < s.N && k < s.K)
              v = overlap_elem(kp, bp, (int64_t)bka[k] + ia_n, (int64_t)bkb[k] + ib_n, s.ket_sig, s.bra_sig, s.phys);
            uint32_t t0[T_P], t1[T_P];
            tn_split3(v.x, -v.y, t0);
            tn_split3(v.y, v.x, t1);
#pragma unroll
            for (int q = 0; q < T_P; ++q) {
              w0[q][i] = t0[q];
              w1[q][i] = t1[q];
            }
          }
#pragma unroll
          for (int q = 0; q < T_P; ++q) {
            sts128(bbase + q * B_BYTES + sw128_off(2 * nl, c16), w0[q]);
            sts128(bbase + q * B_BYTES + sw128_off(2 * nl + 1, c16), w1[q]);
          }
        }
        // generic-proxy writes -> visible to the tensor core (async proxy), then arrive
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bar_arrive(s_u32(&full[st]));
      }
    }
    // ---------------- epilogue (warps 2..5 -> TMEM lane groups 2, 3, 0, 1)
    const bool ok = bar_wait(s_u32(&done), 0u, err, 14);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int lg = warp & 3;
    const int ro = rowoff[lg * 32 + lane];
    const bool all = ok && (*(volatile int *)err == 0);
    const int32_t *ocol = a.tab + s.t_ocol;
#pragma unroll 1
    for (int c0 = 0; c0 < BN && all; c0 += 16) {
      // all accumulators of this 16-column block, one wait, summed smallest first
      uint32_t r[GROUPS][16];
#pragma unroll
      for (int g = 0; g < GROUPS; ++g) {
        const uint32_t taddr = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(g * BN + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[g][0]), "=r"(r[g][1]), "=r"(r[g][2]), "=r"(r[g][3]), "=r"(r[g][4]), "=r"(r[g][5]),
              "=r"(r[g][6]), "=r"(r[g][7]), "=r"(r[g][8]), "=r"(r[g][9]), "=r"(r[g][10]), "=r"(r[g][11]),
              "=r"(r[g][12]), "=r"(r[g][13]), "=r"(r[g][14]), "=r"(r[g][15])
            : "r"(taddr));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float acc[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float v = 0.f;
#pragma unroll
        for (int g = GROUPS - 1; g >= 0; --g)
          if (g >= R || (int64_t)g < nk * 4) v += __uint_as_float(r[g][j]);   // unwritten order-0 slots skipped
        acc[j] = v;
      }
      if (ro >= 0) store_cols8(out, a.t_stride, item, ro, ocol, (nr0 + c0) >> 1, s.N, acc);   // eight complex columns
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// driver entry point for tensor-map encoding (no link-time dependency on libcuda)
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 3-D bf16 map {inner, rows, items}, box {64, box_rows, 1}, 128-byte swizzle, zero fill outside
bool make_map(CUtensorMap *m, const void *base, uint64_t inner, uint64_t rows, uint64_t items, uint64_t row_bytes,
              uint64_t item_bytes, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {inner, rows, items};
  cuuint64_t strides[2] = {row_bytes, item_bytes};
  cuuint32_t box[3] = {64, box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN, int R, int S, int BM>
cudaError_t launch_t(const StepParams &s, const ContractArgs &a, const Pieces &A, const Pieces &B, const OutDesc &out,
                     int *err, const float2 *ket, const float2 *bra, const float2 *cbuf, int64_t c_stride,
                     int64_t c_items, cudaStream_t st) {
  constexpr bool BUILD = BM != 0;
  constexpr size_t stage = (size_t)T_P * (T_BM * 128 + BN * 128);
  // the dynamic shared memory limit on the current device (set once per device)
  const int max_dyn = tn_smem_optin<tma_step_kernel<BN, R, S, BM>>();
  if (max_dyn < 0) return cudaErrorInvalidValue;
  size_t smem = S * stage + 1024;
  if (smem > (size_t)max_dyn) return cudaErrorInvalidValue;
  // BM 1: stage the node tensors in shared memory when they fit beside the stage ring
  const size_t node_bytes = (size_t)(s.phys * s.ket_sig + s.phys * s.bra_sig) * sizeof(float2);
  const int staged = (BM == 1 && smem + node_bytes <= (size_t)max_dyn) ? 1 : 0;
  if (staged) smem += node_bytes;
  CUtensorMap mA[3], mB[3];
  const uint64_t K2 = (uint64_t)(2 * s.K), N2 = (uint64_t)(2 * s.N);
  for (int q = 0; q < T_P; ++q) {
    if (!make_map(&mA[q], (const uint16_t *)A.base + q * A.plane_elems, K2, (uint64_t)s.M, (uint64_t)a.items, K2 * 2,
                  (uint64_t)A.item_elems * 2, T_BM))
      return cudaErrorInvalidValue;
    if (BUILD) {
      mB[q] = mA[q];   // unused: B is built in shared memory
    } else if (!make_map(&mB[q], (const uint16_t *)B.base + q * B.plane_elems, K2, N2, (uint64_t)a.items, K2 * 2,
                         (uint64_t)B.item_elems * 2, BN)) {
      return cudaErrorInvalidValue;
    }
  }
  const int64_t tiles = ((s.M + T_BM - 1) / T_BM) * ((2 * s.N + BN - 1) / BN);
  const int64_t grid = tiles * a.items;
  if (grid <= 0) return cudaSuccess;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  tma_step_kernel<BN, R, S, BM><<<(unsigned)grid, T_THREADS, smem, st>>>(mA[0], mA[1], mA[2], mB[0], mB[1], mB[2], s,
                                                                         a, out, err, ket, bra, cbuf, c_stride,
                                                                         c_items > 0 ? c_items : a.items, staged);
  tn_count_launch(1);
  return cudaGetLastError();
}

}  // namespace

bool tma_step_supported(const StepParams &s) {
  // 16-byte TMA strides (K a multiple of 4), tiles mostly useful, indices within 32 bits
  return s.M >= 64 && 2 * s.N >= 64 && s.K >= 8 && (s.K % 4) == 0 && 2 * s.K < (1LL << 31);
}

cudaError_t launch_step_tma(const StepParams &s, const ContractArgs &a, const Pieces &A, const Pieces &B,
                            const OutDesc &out, int *err, cudaStream_t st, int bn, const float2 *ket,
                            const float2 *bra, const float2 *cbuf, int64_t c_stride, int64_t c_items) {
  if (bn == 0) bn = (2 * s.N >= 128 && s.K < TN_TMA_LONG_K) ? 128 : 64;
  const int bm = cbuf ? 2 : ket ? 1 : 0;
  if (bm == 1 && !bra) return cudaErrorInvalidValue;
#define TN_TMA_LAUNCH(BNV, RV, SV)                                                                     \
  switch (bm) {                                                                                        \
    case 0: return launch_t<BNV, RV, SV, 0>(s, a, A, B, out, err, ket, bra, cbuf, c_stride, c_items, st);       \
    case 1: return launch_t<BNV, RV, SV, 1>(s, a, A, B, out, err, ket, bra, cbuf, c_stride, c_items, st);       \
    default: return launch_t<BNV, RV, SV, 2>(s, a, A, B, out, err, ket, bra, cbuf, c_stride, c_items, st);      \
  }
  if (bn == 128 && 2 * s.N >= 128 && s.K < TN_TMA_LONG_K) { TN_TMA_LAUNCH(128, 3, 2) }
  if (bn == 64) { TN_TMA_LAUNCH(64, 7, 3) }
#undef TN_TMA_LAUNCH
  return cudaErrorInvalidValue;
}

// Persistent TMA-fed tcgen05 contraction step (BF16x6 form), one CTA per SM.
//
// The arithmetic is that of the one-tile-per-CTA step kernel: the same operand pieces, the same
// six products x_i*y_j (i + j <= 2) per 16-real K slice with order 0 spread round-robin over R
// accumulators and orders 1 and 2 in one more, and the same smallest-first sum in the
// epilogue; with the same R (128-column tiles, K > 64) both kernels give the same bits. What
// changes is the schedule. Each CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// (item-major, then 128-row block, then BN-column block) with roles in separate warps:
//   warp 0     TMA producer: per 64-real K chunk of every tile, the pieces that come by TMA (the
//              A pieces unless the input is read as complex64, the B pieces in BM 0) into a
//              ring of S shared-memory stages, and in the complex64-input form (AC) the
//              input's box of fp32 pairs (128 rows x 32 complex) into a separate raw ring; the
//              rings continue across tile boundaries, so the next tile's operands load while
//              this one finishes;
//   warp 1     MMA issuer: tcgen05.mma into accumulator set (tile number mod NBUF); before a
//              tile it waits until the epilogue has drained that set ("tempty"), after it it
//              commits to "tfull";
//   B builders (BM 2, four warps from warp 2): read the overlap operand as complex64 [N][K],
//              split it into bf16 pieces and store them swizzled into each stage;
//   A builders (AC: four warps after the B builders, or eight from warp 2 in BM 0): take the
//              raw box into registers, hand it back, split it into the three pieces and store
//              them swizzled into the stage (the pieces the previous step's epilogue would have
//              written in the pre-split format, so both forms give the same bits, and the
//              previous step writes 8 bytes per value instead of 12);
//   the last four warps, epilogue: wait "tfull", read the accumulators with tcgen05.ld (warp w
//              reads TMEM lanes 32 * (w mod 4) ..), sum, store into the next step's layout,
//              arrive "tempty".
// With NBUF = 2 (64-column tiles: 2 x 4 x 64 TMEM columns; 128-column tiles of a short K, one
// order-0 accumulator: 2 x 2 x 128) the MMAs of one tile run while the epilogue drains the
// previous one; with NBUF = 1 (128-column tiles of a longer K, all 512 columns) the MMAs wait
// only for the drain, not for the CTA's setup, pipeline fill or launch of a next CTA.
// Every wait is bounded by a clock limit; a role that gives up records an error code and
// stops, the others stop at their next wait or tile, and the MMA issuer waits (bounded) for its
// own MMAs before the CTA frees its TMEM.
#pragma once

#include <cstring>

#include "tc_persist.h"
#include "tc_ptx.h"
#include "tn_device.h"

namespace {

using namespace tcx;

// warps: producer, MMA issuer, B builders (four, when B is split from complex64), A builders
// (when A is split from complex64: four beside B builders, else eight), four epilogue warps
constexpr int p_bwarps(int bm) { return bm == 2 ? 4 : 0; }
constexpr int p_awarps(int bm, bool ac) { return ac ? (bm == 2 ? 4 : 8) : 0; }
constexpr int p_threads(int bm, bool ac) { return 32 * (2 + p_bwarps(bm) + p_awarps(bm, ac) + 4); }
// complex64 input boxes (32 KB each) the complex64-A form keeps in flight beside its stage ring
constexpr int p_raw_stages(int bn) { return bn == 128 ? 1 : 2; }
constexpr int P_BM = 128;
constexpr int P_PIECES = 3;
constexpr long long P_WAIT = 500000000LL;   // ~0.25 s at 2 GHz

__device__ __forceinline__ void tile_coords(int64_t t, int64_t tiles_m, int64_t tiles_n, int BN, int &item, int &m0,
                                            int &nr0) {
  const int64_t per_item = tiles_m * tiles_n;
  item = (int)(t / per_item);
  const int64_t rem = t % per_item;
  m0 = (int)((rem / tiles_n) * P_BM);
  nr0 = (int)((rem % tiles_n) * BN);
}

template <int BN, int R, int S, int NBUF, int BM, bool AC>
__global__ void __launch_bounds__(p_threads(BM, AC), 1)
tma_persist_kernel(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
                   const __grid_constant__ CUtensorMap tA2, const __grid_constant__ CUtensorMap tB0,
                   const __grid_constant__ CUtensorMap tB1, const __grid_constant__ CUtensorMap tB2,
                   const __grid_constant__ CUtensorMap tR, StepParams s, ContractArgs a, OutDesc out, int *err,
                   const float2 *cbuf, int64_t c_stride, int64_t c_items) {
  static_assert(BM == 0 || BM == 2, "B loaded by TMA (0) or split from complex64 (2)");
  constexpr bool BUILD = BM != 0;
  constexpr int NBW = p_bwarps(BM), NAW = p_awarps(BM, AC);
  constexpr bool STAGE_TMA = !AC || !BUILD;          // the producer loads pieces into the stages
  // arrivals that complete a stage: the producer's byte-count arrival (when it loads pieces) and
  // one per builder thread
  constexpr uint32_t FULL_COUNT = (STAGE_TMA ? 1 : 0) + 32 * (NBW + NAW);
  constexpr int RAW_S = AC ? p_raw_stages(BN) : 1;    // complex64 input boxes in flight
  constexpr uint32_t RAW_BYTES = P_BM * 64 * 4;
  constexpr int A_BYTES = P_BM * 128, B_BYTES = BN * 128;
  constexpr int STAGE = P_PIECES * (A_BYTES + B_BYTES);
  constexpr int GROUPS = R + 1;                  // R order-0 accumulators + one for orders 1 and 2
  constexpr int SET = GROUPS * BN;               // TMEM columns of one accumulator set
  static_assert(NBUF * SET <= 512, "TMEM columns");
  constexpr uint32_t TMEM_COLS = NBUF * SET <= 32 ? 32 : NBUF * SET <= 64 ? 64 : NBUF * SET <= 128 ? 128
                                 : NBUF * SET <= 256 ? 256 : 512;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[S], empty[S], tfull[NBUF], tempty[NBUF], mdone, rawfull[RAW_S],
      rawempty[RAW_S];
  __shared__ uint32_t tmem_s;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t tiles_m = (s.M + P_BM - 1) / P_BM, tiles_n = (2 * s.N + BN - 1) / BN;
  const int64_t n_tiles = tiles_m * tiles_n * a.items;
  const int64_t nk = (2 * s.K + 63) / 64;        // 64-real K chunks per tile

  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      bar_init(s_u32(&full[i]), FULL_COUNT);
      bar_init(s_u32(&empty[i]), 1);
    }
    for (int i = 0; i < NBUF; ++i) {
      bar_init(s_u32(&tfull[i]), 1);                    // tcgen05.commit
      bar_init(s_u32(&tempty[i]), 128);                 // the 128 epilogue threads
    }
    bar_init(s_u32(&mdone), 1);
    if (AC)
      for (int i = 0; i < RAW_S; ++i) {
        bar_init(s_u32(&rawfull[i]), 1);                // the producer's byte-count arrival
        bar_init(s_u32(&rawempty[i]), 32 * (NAW > 0 ? NAW : 1));   // the A builders
      }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(&tmem_s)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_s;

  uint8_t *const raw = smem + S * STAGE;            // the complex64-A ring (AC only)
  if (warp == 0) {
    // ---------------- TMA producer: per K chunk, the complex64 input box into the raw ring
    // (AC) and the pieces (A unless AC, B unless built) into the stage ring
    if (lane == 0) {
      const CUtensorMap *mA[3] = {&tA0, &tA1, &tA2};
      const CUtensorMap *mB[3] = {&tB0, &tB1, &tB2};
      constexpr uint32_t STAGE_BYTES = (AC ? 0 : P_PIECES * A_BYTES) + (BUILD ? 0 : P_PIECES * B_BYTES);
      int64_t g = 0;                             // chunks issued by this CTA
      bool ok = true;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        if (*(volatile int *)err != 0) break;
        int item, m0, nr0;
        tile_coords(t, tiles_m, tiles_n, BN, item, m0, nr0);
        const int bz = (int)((int64_t)item % c_items);   // the B copy of this item
        for (int64_t kc = 0; kc < nk; ++kc) {
          if (AC) {
            const int rs = (int)(g % RAW_S);
            if (g >= RAW_S && !bar_wait(s_u32(&rawempty[rs]), (uint32_t)(((g / RAW_S) - 1) & 1), err, 39, P_WAIT)) {
              ok = false;
              break;
            }
            bar_expect_tx(s_u32(&rawfull[rs]), RAW_BYTES);
            tma_3d(s_u32(raw + rs * RAW_BYTES), &tR, (int)(kc * 64), m0, item, s_u32(&rawfull[rs]));
          }
          if (STAGE_TMA) {
            const int st = (int)(g % S);
            const uint32_t it = (uint32_t)(g / S);
            if (g >= S && !bar_wait(s_u32(&empty[st]), (it - 1) & 1, err, 31, P_WAIT)) {
              ok = false;
              break;
            }
            uint8_t *base = smem + st * STAGE;
            bar_expect_tx(s_u32(&full[st]), STAGE_BYTES);
            if (!AC)
              for (int q = 0; q < P_PIECES; ++q)
                tma_3d(s_u32(base + q * A_BYTES), mA[q], (int)(kc * 64), m0, item, s_u32(&full[st]));
            if (!BUILD)
              for (int q = 0; q < P_PIECES; ++q)
                tma_3d(s_u32(base + P_PIECES * A_BYTES + q * B_BYTES), mB[q], (int)(kc * 64), nr0, bz,
                       s_u32(&full[st]));
          }
          ++g;
        }
      }
      if (g > 0) {   // the last loads must have landed before the CTA may exit
        if (AC) bar_wait(s_u32(&rawfull[(g - 1) % RAW_S]), (uint32_t)(((g - 1) / RAW_S) & 1), err, 40, P_WAIT);
        if (STAGE_TMA) bar_wait(s_u32(&full[(g - 1) % S]), (uint32_t)(((g - 1) / S) & 1), err, 32, P_WAIT);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(P_BM, BN);
      int64_t g = 0, tl = 0;                     // chunks consumed, tiles started by this CTA
      bool ok = true;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++tl) {
        if (*(volatile int *)err != 0) break;
        const int buf = (int)(tl % NBUF);
        if (tl >= NBUF && !bar_wait(s_u32(&tempty[buf]), (uint32_t)(((tl / NBUF) - 1) & 1), err, 33, P_WAIT)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(buf * SET);
        for (int64_t kc = 0; kc < nk; ++kc) {
          const int st = (int)(g % S);
          if (!bar_wait(s_u32(&full[st]), (uint32_t)((g / S) & 1), err, 34, P_WAIT)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = s_u32(smem + st * STAGE), b0 = a0 + P_PIECES * A_BYTES;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {        // 16 bf16 (32 bytes) of K per instruction
            const uint32_t off = (uint32_t)ks * 32u;
            const int64_t q = kc * 4 + ks;
            const uint32_t first = (q == 0) ? 0u : 1u;
            mma_bf16(acc + (uint32_t)((q % R) * BN), desc_sw128(a0 + off), desc_sw128(b0 + off), idesc,
                     q < R ? 0u : 1u);
            mma_bf16(acc + (uint32_t)(R * BN), desc_sw128(a0 + off), desc_sw128(b0 + B_BYTES + off), idesc, first);
            mma_bf16(acc + (uint32_t)(R * BN), desc_sw128(a0 + A_BYTES + off), desc_sw128(b0 + off), idesc, 1u);
            mma_bf16(acc + (uint32_t)(R * BN), desc_sw128(a0 + off), desc_sw128(b0 + 2 * B_BYTES + off), idesc, 1u);
            mma_bf16(acc + (uint32_t)(R * BN), desc_sw128(a0 + A_BYTES + off), desc_sw128(b0 + B_BYTES + off),
                     idesc, 1u);
            mma_bf16(acc + (uint32_t)(R * BN), desc_sw128(a0 + 2 * A_BYTES + off), desc_sw128(b0 + off), idesc, 1u);
          }
          mma_commit_to(s_u32(&empty[st]));
          ++g;
        }
        if (!ok) break;
        mma_commit_to(s_u32(&tfull[buf]));
      }
      // every MMA this thread issued has completed before the CTA frees its TMEM
      mma_commit_to(s_u32(&mdone));
      bar_wait(s_u32(&mdone), 0u, err, 35, P_WAIT);
    }
  } else if (BUILD && warp < 2 + NBW) {
    // ---------------- B builders (BM 2): tile rows nr0 .. nr0 + BN - 1 of the real embedding
    // (complex column n = row / 2; row 2n = (Re c, -Im c), row 2n + 1 = (Im c, Re c) along k),
    // reals kc*64 .. kc*64 + 63 (complex k = kc*32 .. kc*32 + 31); zeros outside K and N
    if (BUILD) {
      const int bt = tid - 64;
      constexpr int TASKS = (BN / 2) * 8 / 128;   // tasks: four consecutive complex k of one column
      int64_t g = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        if (*(volatile int *)err != 0) break;
        int item, m0, nr0;
        tile_coords(t, tiles_m, tiles_n, BN, item, m0, nr0);
        const int64_t n_base = nr0 >> 1;
        const float2 *cb = cbuf + ((int64_t)item % c_items) * c_stride;
        float4 xn[TASKS][2];
        auto load = [&](int64_t kc, float4 (&x)[TASKS][2]) {
#pragma unroll
          for (int j = 0; j < TASKS; ++j) {
            const int u = bt + 128 * j, c16 = u & 7, nl = u >> 3;
            const int64_t n = n_base + nl, k0 = kc * 32 + c16 * 4;
            x[j][0] = x[j][1] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (n < s.N && k0 < s.K) {   // K % 4 == 0: the four k are all in range or all out
              const float4 *src = reinterpret_cast<const float4 *>(cb + n * s.K + k0);
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
          const int st = (int)(g % S);
          const uint32_t it = (uint32_t)(g / S);
          if (g >= S && !bar_wait(s_u32(&empty[st]), (it - 1) & 1, err, 36, P_WAIT)) {
            ok = false;
            break;
          }
          const uint32_t bbase = s_u32(smem + st * STAGE + P_PIECES * A_BYTES);
#pragma unroll
          for (int j = 0; j < TASKS; ++j) {
            const int u = bt + 128 * j, c16 = u & 7, nl = u >> 3;
            const float re[4] = {x[j][0].x, x[j][0].z, x[j][1].x, x[j][1].z};
            const float im[4] = {x[j][0].y, x[j][0].w, x[j][1].y, x[j][1].w};
            uint32_t w0[P_PIECES][4], w1[P_PIECES][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              uint32_t t0[P_PIECES], t1[P_PIECES];
              tn_split3(re[i], -im[i], t0);
              tn_split3(im[i], re[i], t1);
#pragma unroll
              for (int q = 0; q < P_PIECES; ++q) {
                w0[q][i] = t0[q];
                w1[q][i] = t1[q];
              }
            }
#pragma unroll
            for (int q = 0; q < P_PIECES; ++q) {
              sts128(bbase + q * B_BYTES + sw128_off(2 * nl, c16), w0[q]);
              sts128(bbase + q * B_BYTES + sw128_off(2 * nl + 1, c16), w1[q]);
            }
          }
          // generic-proxy writes -> visible to the tensor core (async proxy), then arrive
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          bar_arrive(s_u32(&full[st]));
          ++g;
        }
      }
    }
  } else if (AC && warp < 2 + NBW + NAW) {
    // ---------------- A builders (complex64 A): the box of chunk g holds tile rows m0 .. m0 + 127,
    // complex k = kc*32 .. kc*32 + 31 as (re, im) fp32 pairs, 256 bytes a row, zeros outside M and
    // K. Task u: row u / 8, 16-byte piece chunk u % 8 of the row (four complex k). The values are
    // taken into registers and the box handed back before the stage is written.
    constexpr int AT = 32 * (NAW > 0 ? NAW : 4);  // A-builder threads (the branch is dead without AC)
    const int at = tid - 32 * (2 + NBW);
    constexpr int ATASKS = P_BM * 8 / AT;
    int64_t g = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      if (*(volatile int *)err != 0) break;
      for (int64_t kc = 0; kc < nk; ++kc) {
        const int rs = (int)(g % RAW_S);
        if (!bar_wait(s_u32(&rawfull[rs]), (uint32_t)((g / RAW_S) & 1), err, 41, P_WAIT)) {
          ok = false;
          break;
        }
        const uint32_t rbase = s_u32(raw + rs * RAW_BYTES);
        float4 x[ATASKS][2];
#pragma unroll
        for (int j = 0; j < ATASKS; ++j) {
          const int u = at + AT * j, c16 = u & 7, r = u >> 3;
          const uint32_t src = rbase + (uint32_t)(r * 256 + c16 * 32);
          asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                       : "=f"(x[j][0].x), "=f"(x[j][0].y), "=f"(x[j][0].z), "=f"(x[j][0].w)
                       : "r"(src)
                       : "memory");
          asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                       : "=f"(x[j][1].x), "=f"(x[j][1].y), "=f"(x[j][1].z), "=f"(x[j][1].w)
                       : "r"(src + 16u)
                       : "memory");
        }
        // the box may be overwritten by the next TMA load (async proxy) once all have read it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bar_arrive(s_u32(&rawempty[rs]));
        const int st = (int)(g % S);
        const uint32_t it = (uint32_t)(g / S);
        if (g >= S && !bar_wait(s_u32(&empty[st]), (it - 1) & 1, err, 38, P_WAIT)) {
          ok = false;
          break;
        }
        const uint32_t abase = s_u32(smem + st * STAGE);
#pragma unroll
        for (int j = 0; j < ATASKS; ++j) {
          const int u = at + AT * j, c16 = u & 7, r = u >> 3;
          const float re[4] = {x[j][0].x, x[j][0].z, x[j][1].x, x[j][1].z};
          const float im[4] = {x[j][0].y, x[j][0].w, x[j][1].y, x[j][1].w};
          uint32_t w[P_PIECES][4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            uint32_t t0[P_PIECES];
            tn_split3(re[i], im[i], t0);
#pragma unroll
            for (int q = 0; q < P_PIECES; ++q) w[q][i] = t0[q];
          }
#pragma unroll
          for (int q = 0; q < P_PIECES; ++q) sts128(abase + q * A_BYTES + sw128_off(r, c16), w[q]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bar_arrive(s_u32(&full[st]));
        ++g;
      }
    }
  } else {
    // ---------------- epilogue (the last four warps; warp w reads TMEM lanes 32 * (w mod 4) ..)
    const int lg = warp & 3;
    const int32_t *ocol = a.tab + s.t_ocol;
    int64_t tl = 0;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++tl) {
      int item, m0, nr0;
      tile_coords(t, tiles_m, tiles_n, BN, item, m0, nr0);
      const int64_t m = m0 + lg * 32 + lane;
      const int ro = m < s.M ? orow_of(s, m) : -1;
      const int buf = (int)(tl % NBUF);
      if (!bar_wait(s_u32(&tfull[buf]), (uint32_t)((tl / NBUF) & 1), err, 37, P_WAIT)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const bool store = *(volatile int *)err == 0;
      const uint32_t acc = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(buf * SET);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        // all accumulators of this 16-column block, one wait, summed smallest first
        uint32_t r[GROUPS][16];
#pragma unroll
        for (int gr = 0; gr < GROUPS; ++gr) tmem_ld16(acc + (uint32_t)(gr * BN + c0), r[gr]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float x = 0.f;
#pragma unroll
          for (int gr = GROUPS - 1; gr >= 0; --gr)
            if (gr >= R || (int64_t)gr < nk * 4) x += __uint_as_float(r[gr][j]);   // unwritten order-0 sets skipped
          v[j] = x;
        }
        if (store && ro >= 0) store_cols8(out, a.t_stride, item, ro, ocol, (nr0 + c0) >> 1, s.N, v);
      }
      // this set's TMEM reads are complete (wait::ld above): hand it back to the MMA issuer
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      bar_arrive(s_u32(&tempty[buf]));
      if (!store) break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    return (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                    cudaSuccess &&
                q == cudaDriverEntryPointSuccess)
               ? reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p)
               : nullptr;
  }();
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
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D fp32 map of a complex64 intermediate {2K reals, rows, items}, box {64, 128, 1}, no
// swizzle, zero fill outside
bool make_map_raw(CUtensorMap *m, const void *base, uint64_t inner, uint64_t rows, uint64_t items, uint64_t row_bytes,
                  uint64_t item_bytes) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {inner, rows, items};
  cuuint64_t strides[2] = {row_bytes, item_bytes};
  cuuint32_t box[3] = {64, P_BM, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int R, int S, int NBUF, int BM, bool AC>
cudaError_t launch_p(const StepParams &s, const ContractArgs &a, const Pieces &A, const Pieces &B, const OutDesc &out,
                     int *err, const float2 *cbuf, int64_t c_stride, int64_t c_items, const float2 *ain,
                     cudaStream_t st) {
  constexpr size_t stage = (size_t)P_PIECES * (P_BM * 128 + BN * 128);
  // the dynamic shared memory limit on the current device (set once per device), and its SM count
  const int max_dyn = tn_smem_optin<tma_persist_kernel<BN, R, S, NBUF, BM, AC>>();
  const int64_t cb_items = c_items > 0 ? c_items : a.items;   // distinct B copies
  int sms = -1;
  {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      sms = n;
  }
  if (max_dyn < 0 || sms <= 0) return cudaErrorInvalidValue;
  const size_t smem = S * stage + (AC ? (size_t)p_raw_stages(BN) * P_BM * 64 * 4 : 0) + 1024;
  if (smem > (size_t)max_dyn) return cudaErrorInvalidValue;
  if (BM == 2 && (!cbuf || c_stride < s.N * s.K)) return cudaErrorInvalidValue;
  if (AC && (!ain || a.t_stride % 2 != 0)) return cudaErrorInvalidValue;   // 16-byte aligned item strides
  CUtensorMap mA[3], mB[3], mR;
  std::memset(&mR, 0, sizeof(CUtensorMap));
  if (AC && !make_map_raw(&mR, ain, (uint64_t)(2 * s.K), (uint64_t)s.M, (uint64_t)a.items, (uint64_t)(2 * s.K) * 4,
                          (uint64_t)a.t_stride * 8))
    return cudaErrorInvalidValue;
  const uint64_t K2 = (uint64_t)(2 * s.K), N2 = (uint64_t)(2 * s.N);
  for (int q = 0; q < P_PIECES; ++q) {
    if (AC) {
      std::memset(&mA[q], 0, sizeof(CUtensorMap));   // unused: A is split from complex64 on chip
    } else if (!make_map(&mA[q], (const uint16_t *)A.base + q * A.plane_elems, K2, (uint64_t)s.M, (uint64_t)a.items,
                         K2 * 2, (uint64_t)A.item_elems * 2, P_BM)) {
      return cudaErrorInvalidValue;
    }
    if (BM == 2) {
      std::memset(&mB[q], 0, sizeof(CUtensorMap));   // unused: B is split from complex64 on chip
    } else if (!make_map(&mB[q], (const uint16_t *)B.base + q * B.plane_elems, K2, N2, (uint64_t)cb_items, K2 * 2,
                         (uint64_t)B.item_elems * 2, BN)) {
      return cudaErrorInvalidValue;
    }
  }
  const int64_t n_tiles = ((s.M + P_BM - 1) / P_BM) * ((2 * s.N + BN - 1) / BN) * a.items;
  if (n_tiles <= 0) return cudaSuccess;
  const int grid = (int)(n_tiles < sms ? n_tiles : sms);
  tma_persist_kernel<BN, R, S, NBUF, BM, AC><<<grid, p_threads(BM, AC), smem, st>>>(
      mA[0], mA[1], mA[2], mB[0], mB[1], mB[2], mR, s, a, out, err, cbuf, c_stride, cb_items);
  tn_count_launch(1);
  return cudaGetLastError();
}

// The launches of one overlap-operand mode BM (the input as pieces or as complex64, at 128- or
// 64-column tiles); each translation unit instantiates one BM.
template <int BM>
cudaError_t persist_dispatch(const StepParams &s, const ContractArgs &a, const Pieces &A, const Pieces &B,
                             const OutDesc &out, int *err, cudaStream_t st, int bn, const float2 *cbuf,
                             int64_t c_stride, int64_t c_items, const float2 *ain) {
  if (!tma_step_supported(s)) return cudaErrorInvalidValue;
  if ((BM == 2) != (cbuf != nullptr)) return cudaErrorInvalidValue;
  if (bn == 0) bn = 2 * s.N >= 128 ? 128 : 64;
#define TN_P_LAUNCH(BNV, RV, SV, SCV, NB)                                                                   \
  return ain ? launch_p<BNV, RV, SCV, NB, BM, true>(s, a, A, B, out, err, cbuf, c_stride, c_items, ain, st) \
             : launch_p<BNV, RV, SV, NB, BM, false>(s, a, A, B, out, err, cbuf, c_stride, c_items, ain, st);
  // short K (at most 8 MMAs of K 16 per accumulator): one order-0 accumulator, so two
  // accumulator sets fit TMEM and the epilogue of one tile overlaps the MMAs of the next
  if (bn == 128 && 2 * s.N >= 128 && 2 * s.K <= 128) { TN_P_LAUNCH(128, 1, 2, 2, 2) }
  if (bn == 128 && 2 * s.N >= 128) { TN_P_LAUNCH(128, 3, 2, 2, 1) }
  if (bn == 64) { TN_P_LAUNCH(64, 3, 3, 2, 2) }
#undef TN_P_LAUNCH
  return cudaErrorInvalidValue;
}

}  // namespace

// Path-ordered contraction of the overlap network, batched over
// (bitstring, slice) items: the first node's C tensor, one SIMT complex GEMM
// per absorption step, and the FP64 sum over slices.
//
// The overlap tensor C^i = sum_sigma A^sigma (ket) B^sigma (bra) of Eq. overlap
// is never stored by the SIMT kernels: each GEMM forms its B operand tile on
// the fly from the node's ket and bra tensors through per-step offset tables,
// with the cut legs fixed by the item's slice. Every intermediate is written by
// its producer directly in the row-major [M][K] layout its consumer reads
// (output offset orow(m) + ocol[n]), so the transposes of a
// transpose-transpose-GEMM step cost no extra pass over memory.
#include <cuda_runtime.h>

#include "tn_device.h"
#include "tn_internal.h"

namespace {

template <typename R> struct C2T;
template <> struct C2T<double> { using T = double2; };
template <> struct C2T<float> { using T = float2; };

template <typename R>
__global__ void form_kernel(StepParams s, ContractArgs a, const typename C2T<R>::T *ket,
                            const typename C2T<R>::T *bra, OutDesc out) {
  using V = typename C2T<R>::T;
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.items * s.N) return;
  int64_t item = idx / s.N, n = idx % s.N;
  ItemCtx c = item_ctx(a, s, item);
  const V *kp = ket + s.ket_off + c.sa;
  const V *bp = bra + c.b * a.bra_stride + s.bra_off + c.sb;
  store_out(out, a.t_stride, item, a.tab[s.t_ocol + n],
            overlap_elem(kp, bp, a.tab[s.t_bna + n], a.tab[s.t_bnb + n], s.ket_sig, s.bra_sig, s.phys));
}

// the overlap tensor in its real embedding B_r[2N][2K] (row 2n = (Re c, -Im c), row 2n+1 =
// (Im c, Re c) along k), as three bf16 planes, for the TMA-fed tensor-core step
__global__ void form_b_kernel(StepParams s, ContractArgs a, const float2 *ket, const float2 *bra, Pieces B,
                              int64_t item0) {
  const unsigned kn = (unsigned)(s.K * s.N), K = (unsigned)s.K;
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t item = item0 + blockIdx.y;
  if (r >= kn) return;
  const unsigned n = r / K, k = r % K;
  ItemCtx c = item_ctx(a, s, item);
  const float2 *kp = ket + s.ket_off + c.sa;
  const float2 *bp = bra + c.b * a.bra_stride + s.bra_off + c.sb;
  const float2 v = overlap_elem(kp, bp, (int64_t)a.tab[s.t_bka + k] + a.tab[s.t_bna + n],
                                (int64_t)a.tab[s.t_bkb + k] + a.tab[s.t_bnb + n], s.ket_sig, s.bra_sig, s.phys);
  uint32_t w0[3], w1[3];
  tn_split3(v.x, -v.y, w0);
  tn_split3(v.y, v.x, w1);
  uint32_t *base = reinterpret_cast<uint32_t *>(const_cast<void *>(B.base)) + item * (B.item_elems / 2);
  const int64_t plane = B.plane_elems / 2, row0 = (int64_t)(2 * n) * K + k, row1 = row0 + K;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    base[q * plane + row0] = w0[q];
    base[q * plane + row1] = w1[q];
  }
}

// the overlap tensor of the absorbed node, per item, as [N][K] complex64 (K contiguous)
__global__ void form_c_kernel(StepParams s, ContractArgs a, const float2 *ket, const float2 *bra, float2 *cbuf,
                              int64_t c_stride, int64_t item0) {
  const unsigned kn = (unsigned)(s.K * s.N), K = (unsigned)s.K;
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;   // element within one item
  const int64_t item = item0 + blockIdx.y;
  if (r >= kn) return;
  const unsigned n = r / K, k = r % K;
  ItemCtx c = item_ctx(a, s, item);
  const float2 *kp = ket + s.ket_off + c.sa;
  const float2 *bp = bra + c.b * a.bra_stride + s.bra_off + c.sb;
  cbuf[item * c_stride + r] = overlap_elem(kp, bp, (int64_t)a.tab[s.t_bka + k] + a.tab[s.t_bna + n],
                                           (int64_t)a.tab[s.t_bkb + k] + a.tab[s.t_bnb + n], s.ket_sig, s.bra_sig, s.phys);
}

// The same overlap tensor with the node's ket and bra tensors staged in shared memory first (they
// are small for most steps): every element then reads shared memory instead of chasing table
// offsets into global memory. Each CTA forms FORM_E * 256 consecutive elements of one item.
constexpr int FORM_E = 8;
__global__ void __launch_bounds__(256)
form_c_smem_kernel(StepParams s, ContractArgs a, const float2 *ket, const float2 *bra, float2 *cbuf,
                   int64_t c_stride, int64_t tk, int64_t tb, int64_t item0) {
  extern __shared__ float2 nodes[];   // tk ket elements, then tb bra elements
  const int64_t item = item0 + blockIdx.y;
  const ItemCtx c = item_ctx(a, s, item);
  const float2 *kg = ket + s.ket_off;
  const float2 *bg = bra + c.b * a.bra_stride + s.bra_off;
  for (int64_t i = threadIdx.x; i < tk; i += 256) nodes[i] = kg[i];
  for (int64_t i = threadIdx.x; i < tb; i += 256) nodes[tk + i] = bg[i];
  __syncthreads();
  const float2 *kp = nodes + c.sa, *bp = nodes + tk + c.sb;
  const int64_t K = s.K, kn = s.K * s.N;
  const int64_t r0 = (int64_t)blockIdx.x * (256 * FORM_E) + threadIdx.x;
#pragma unroll 4
  for (int e = 0; e < FORM_E; ++e) {
    const int64_t r = r0 + (int64_t)e * 256;
    if (r >= kn) break;
    const int64_t n = r / K, k = r % K;
    cbuf[item * c_stride + r] = overlap_elem(kp, bp, (int64_t)a.tab[s.t_bka + k] + a.tab[s.t_bna + n],
                                             (int64_t)a.tab[s.t_bkb + k] + a.tab[s.t_bnb + n], s.ket_sig, s.bra_sig,
                                             s.phys);
  }
}

// Tiled SIMT complex GEMM: one CTA per (item, BM x BN output tile).
template <typename R, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
step_kernel(StepParams s, ContractArgs a, const typename C2T<R>::T *ket, const typename C2T<R>::T *bra,
            const typename C2T<R>::T *tin, OutDesc out) {
  using V = typename C2T<R>::T;
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ V As[BK][BM + 1];
  __shared__ V Bs[BK][BN];
  __shared__ int rowoff[BM];
  const int tid = threadIdx.x;
  const int64_t tiles_m = (s.M + BM - 1) / BM, tiles_n = (s.N + BN - 1) / BN;
  const int64_t blk = blockIdx.x;
  const int64_t item = blk / (tiles_m * tiles_n);
  const int64_t rem = blk % (tiles_m * tiles_n);
  const int64_t m0 = (rem / tiles_n) * BM, n0 = (rem % tiles_n) * BN;
  ItemCtx c = item_ctx(a, s, item);
  const V *kp = ket + s.ket_off + c.sa;
  const V *bp = bra + c.b * a.bra_stride + s.bra_off + c.sb;
  const V *tp = tin + item * a.t_stride;
  const int32_t *bka = a.tab + s.t_bka, *bkb = a.tab + s.t_bkb;
  const int32_t *bna = a.tab + s.t_bna, *bnb = a.tab + s.t_bnb, *ocol = a.tab + s.t_ocol;

  for (int mm = tid; mm < BM; mm += NT) {     // output row offsets
    const int64_t m = m0 + mm;
    rowoff[mm] = m < s.M ? orow_of(s, m) : -1;
  }
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  V acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = cz<V>();
  __syncthreads();

  for (int64_t k0 = 0; k0 < s.K; k0 += BK) {
    for (int idx = tid; idx < BM * BK; idx += NT) {
      int mm = idx / BK, kk = idx % BK;
      int64_t k = k0 + kk, m = m0 + mm;
      As[kk][mm] = (m < s.M && k < s.K) ? tp[m * s.K + k] : cz<V>();
    }
    for (int idx = tid; idx < BK * BN; idx += NT) {
      int kk = idx / BN, nn = idx % BN;
      int64_t k = k0 + kk, n = n0 + nn;
      V v = cz<V>();
      if (k < s.K && n < s.N)
        v = overlap_elem(kp, bp, (int64_t)bka[k] + bna[n], (int64_t)bkb[k] + bnb[n], s.ket_sig, s.bra_sig, s.phys);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      V af[TM], bf[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) af[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bf[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = cfma(af[i], bf[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int ro = rowoff[ty * TM + i];
    if (ro < 0) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      int64_t n = n0 + tx * TN + j;
      if (n < s.N) store_out(out, a.t_stride, item, ro + ocol[n], acc[i][j]);
    }
  }
}

// Small outputs (M*N <= 256, e.g. the last steps): one CTA per item, one warp per output at a
// time, each reducing over K with its lanes and a shuffle tree (no block barriers).
template <typename R>
__global__ void __launch_bounds__(256)
step_small_kernel(StepParams s, ContractArgs a, const typename C2T<R>::T *ket, const typename C2T<R>::T *bra,
                  const typename C2T<R>::T *tin, OutDesc out, int staged) {
  using V = typename C2T<R>::T;
  extern __shared__ unsigned char small_nodes_raw[];
  const int64_t item = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  ItemCtx c = item_ctx(a, s, item);
  const V *kp = ket + s.ket_off + c.sa;
  const V *bp = bra + c.b * a.bra_stride + s.bra_off + c.sb;
  if (staged) {   // the node's tensors (small) in shared memory first
    V *nodes = reinterpret_cast<V *>(small_nodes_raw);
    const int64_t tk = s.phys * s.ket_sig, tb = s.phys * s.bra_sig;
    const V *kg = ket + s.ket_off, *bg = bra + c.b * a.bra_stride + s.bra_off;
    for (int64_t i = threadIdx.x; i < tk; i += 256) nodes[i] = kg[i];
    for (int64_t i = threadIdx.x; i < tb; i += 256) nodes[tk + i] = bg[i];
    __syncthreads();
    kp = nodes + c.sa;
    bp = nodes + tk + c.sb;
  }
  const V *tp = tin + item * a.t_stride;
  const int32_t *bka = a.tab + s.t_bka, *bkb = a.tab + s.t_bkb;
  const int32_t *bna = a.tab + s.t_bna, *bnb = a.tab + s.t_bnb, *ocol = a.tab + s.t_ocol;
  for (int64_t oi = warp; oi < s.M * s.N; oi += 8) {
    const int64_t m = oi / s.N, n = oi % s.N;
    V acc = cz<V>();
    for (int64_t k = lane; k < s.K; k += 32) {
      V cv = overlap_elem(kp, bp, (int64_t)bka[k] + bna[n], (int64_t)bkb[k] + bnb[n], s.ket_sig, s.bra_sig, s.phys);
      acc = cfma(tp[m * s.K + k], cv, acc);
    }
    for (int o = 16; o; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) store_out(out, a.t_stride, item, orow_of(s, m) + ocol[n], acc);
  }
}

// Few rows, many columns (M <= 16, M * K <= 2048): the item's M x K input block sits in shared memory
// and each thread forms its column n of the overlap tensor on the fly and writes M outputs.
template <typename R>
__global__ void __launch_bounds__(256)
step_narrow_kernel(StepParams s, ContractArgs a, const typename C2T<R>::T *ket, const typename C2T<R>::T *bra,
                   const typename C2T<R>::T *tin, OutDesc out) {
  using V = typename C2T<R>::T;
  __shared__ V Ts[2048];
  const int64_t ctas_n = (s.N + 255) / 256;
  const int64_t item = blockIdx.x / ctas_n;
  const int64_t n = (blockIdx.x % ctas_n) * 256 + threadIdx.x;
  ItemCtx c = item_ctx(a, s, item);
  const V *tp = tin + item * a.t_stride;
  const int MK = (int)(s.M * s.K);
  for (int i = threadIdx.x; i < MK; i += 256) Ts[i] = tp[i];
  __syncthreads();
  if (n >= s.N) return;
  const V *kp = ket + s.ket_off + c.sa;
  const V *bp = bra + c.b * a.bra_stride + s.bra_off + c.sb;
  const int32_t *bka = a.tab + s.t_bka, *bkb = a.tab + s.t_bkb;
  const int64_t ia_n = a.tab[s.t_bna + n], ib_n = a.tab[s.t_bnb + n];
  V acc[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) acc[m] = cz<V>();
  for (int64_t k = 0; k < s.K; ++k) {
    const V cv = overlap_elem(kp, bp, (int64_t)bka[k] + ia_n, (int64_t)bkb[k] + ib_n, s.ket_sig, s.bra_sig, s.phys);
#pragma unroll
    for (int m = 0; m < 16; ++m)
      if (m < s.M) acc[m] = cfma(Ts[m * s.K + k], cv, acc[m]);
  }
  const int oc = a.tab[s.t_ocol + n];
#pragma unroll
  for (int m = 0; m < 16; ++m)
    if (m < s.M) store_out(out, a.t_stride, item, orow_of(s, m) + oc, acc[m]);
}

// Streaming step for small K and N (K, N <= 16) and many rows: the item's C tile sits in shared
// memory, each thread reads its row of T_in (K contiguous complex) and writes N outputs.
template <typename R>
__global__ void __launch_bounds__(256)
step_stream_kernel(StepParams s, ContractArgs a, const typename C2T<R>::T *ket, const typename C2T<R>::T *bra,
                   const typename C2T<R>::T *tin, OutDesc out, int64_t rows_per_cta) {
  using V = typename C2T<R>::T;
  __shared__ V Cs[16 * 16];
  __shared__ int oc[16];
  const int tid = threadIdx.x;
  const int64_t ctas_m = (s.M + rows_per_cta - 1) / rows_per_cta;
  const int64_t item = blockIdx.x / ctas_m;
  const int64_t m0 = (blockIdx.x % ctas_m) * rows_per_cta;
  ItemCtx c = item_ctx(a, s, item);
  const V *kp = ket + s.ket_off + c.sa;
  const V *bp = bra + c.b * a.bra_stride + s.bra_off + c.sb;
  const int K = (int)s.K, N = (int)s.N;
  if (tid < K * N) {
    const int k = tid / N, n = tid % N;
    Cs[tid] = overlap_elem(kp, bp, (int64_t)a.tab[s.t_bka + k] + a.tab[s.t_bna + n],
                           (int64_t)a.tab[s.t_bkb + k] + a.tab[s.t_bnb + n], s.ket_sig, s.bra_sig, s.phys);
  }
  if (tid < N) oc[tid] = a.tab[s.t_ocol + tid];
  __syncthreads();
  const V *tp = tin + item * a.t_stride;
  const int64_t m1 = m0 + rows_per_cta < s.M ? m0 + rows_per_cta : s.M;
  const bool four = (N == 4 && oc[1] == oc[0] + 1 && oc[2] == oc[0] + 2 && oc[3] == oc[0] + 3);   // consecutive
  for (int64_t m = m0 + tid; m < m1; m += 256) {
    V x[16];
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (k < K) x[k] = tp[m * K + k];
    const int ro = orow_of(s, m);
    if (four) {
      R v[8];
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        V acc = cz<V>();
#pragma unroll
        for (int k = 0; k < 16; ++k)
          if (k < K) acc = cfma(x[k], Cs[k * 4 + n], acc);
        v[2 * n] = acc.x;
        v[2 * n + 1] = acc.y;
      }
      store_out4(out, a.t_stride, item, ro + oc[0], v);
      continue;
    }
#pragma unroll
    for (int n = 0; n < 16; ++n) {
      if (n >= N) break;
      V acc = cz<V>();
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (k < K) acc = cfma(x[k], Cs[k * N + n], acc);
      store_out(out, a.t_stride, item, ro + oc[n], acc);
    }
  }
}

// The same streaming step with K and N fixed at compile time (small register footprint): a
// thread holds its row of T_in in registers (16-byte loads for complex64 when K is even), and
// each group of four columns whose outputs are adjacent in the next layout goes out as one
// four-wide store.
template <typename R, int KK, int NN>
__global__ void __launch_bounds__(256)
step_stream_fixed(StepParams s, ContractArgs a, const typename C2T<R>::T *ket, const typename C2T<R>::T *bra,
                  const typename C2T<R>::T *tin, OutDesc out, int64_t rows_per_cta) {
  using V = typename C2T<R>::T;
  constexpr int NQ = (NN + 3) / 4;
  __shared__ V Cs[KK * NN];
  __shared__ int oc[NN];
  __shared__ int four[NQ];
  const int tid = threadIdx.x;
  const int64_t ctas_m = (s.M + rows_per_cta - 1) / rows_per_cta;
  const int64_t item = blockIdx.x / ctas_m;
  const int64_t m0 = (blockIdx.x % ctas_m) * rows_per_cta;
  ItemCtx c = item_ctx(a, s, item);
  {
    const V *kp = ket + s.ket_off + c.sa;
    const V *bp = bra + c.b * a.bra_stride + s.bra_off + c.sb;
    for (int i = tid; i < KK * NN; i += 256) {
      const int k = i / NN, n = i - k * NN;
      Cs[i] = overlap_elem(kp, bp, (int64_t)a.tab[s.t_bka + k] + a.tab[s.t_bna + n],
                           (int64_t)a.tab[s.t_bkb + k] + a.tab[s.t_bnb + n], s.ket_sig, s.bra_sig, s.phys);
    }
  }
  if (tid < NN) oc[tid] = a.tab[s.t_ocol + tid];
  __syncthreads();
  if (tid < NQ) {   // columns 4q .. 4q + 3 land on consecutive offsets
    bool f = NN % 4 == 0;
    if (f)
      for (int j = 1; j < 4; ++j) f = f && oc[4 * tid + j] == oc[4 * tid] + j;
    four[tid] = f;
  }
  __syncthreads();
  const V *tp = tin + item * a.t_stride;
  const int64_t m1 = m0 + rows_per_cta < s.M ? m0 + rows_per_cta : s.M;
  for (int64_t m = m0 + tid; m < m1; m += 256) {
    V x[KK];
    if constexpr (sizeof(V) == 8 && KK % 2 == 0) {
      const float4 *src = reinterpret_cast<const float4 *>(tp + m * KK);
#pragma unroll
      for (int k = 0; k < KK; k += 2) {
        const float4 q = src[k / 2];
        x[k].x = q.x;
        x[k].y = q.y;
        x[k + 1].x = q.z;
        x[k + 1].y = q.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < KK; ++k) x[k] = tp[m * KK + k];
    }
    const int ro = orow_of(s, m);
    R v[2 * NN];
#pragma unroll
    for (int n = 0; n < NN; ++n) {
      V acc = cz<V>();
#pragma unroll
      for (int k = 0; k < KK; ++k) acc = cfma(x[k], Cs[k * NN + n], acc);
      v[2 * n] = acc.x;
      v[2 * n + 1] = acc.y;
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      if (NN % 4 == 0 && four[q]) {
        store_out4(out, a.t_stride, item, ro + oc[4 * q], v + 8 * q);
      } else {
#pragma unroll
        for (int n = 4 * q; n < 4 * q + 4 && n < NN; ++n) {
          V t;
          t.x = v[2 * n];
          t.y = v[2 * n + 1];
          store_out(out, a.t_stride, item, ro + oc[n], t);
        }
      }
    }
  }
}

template <typename R, int KK, int NN>
cudaError_t launch_stream_fixed(const StepParams &s, const ContractArgs &a, const void *ket, const void *bra,
                                const void *t_in, const OutDesc &t_out, cudaStream_t st) {
  using V = typename C2T<R>::T;
  const int64_t rows = 1024;
  const int64_t grid = ((s.M + rows - 1) / rows) * a.items;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  step_stream_fixed<R, KK, NN><<<(unsigned)grid, 256, 0, st>>>(s, a, (const V *)ket, (const V *)bra,
                                                                (const V *)t_in, t_out, rows);
  tn_count_launch(1);
  return cudaGetLastError();
}

template <typename R>
__global__ void slice_sum_kernel(const typename C2T<R>::T *res, int64_t stride, int64_t n_bits, int64_t n_slices,
                                 int accumulate, double2 *out) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_bits) return;
  double sr = 0, si = 0;
  if (accumulate) { sr = out[b].x; si = out[b].y; }
  for (int64_t sl = 0; sl < n_slices; ++sl) {   // fixed order, FP64
    auto v = res[(b * n_slices + sl) * stride];
    sr += (double)v.x;
    si += (double)v.y;
  }
  out[b] = make_double2(sr, si);
}

template <typename R, int BM, int BN, int BK, int TM, int TN>
cudaError_t launch_tiled(const StepParams &s, const ContractArgs &a, const void *ket, const void *bra,
                         const void *t_in, const OutDesc &t_out, cudaStream_t st) {
  using V = typename C2T<R>::T;
  int64_t tiles = ((s.M + BM - 1) / BM) * ((s.N + BN - 1) / BN);
  int64_t grid = tiles * a.items;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  step_kernel<R, BM, BN, BK, TM, TN><<<(unsigned)grid, (BM / TM) * (BN / TN), 0, st>>>(
      s, a, (const V *)ket, (const V *)bra, (const V *)t_in, t_out);
  tn_count_launch(1);
  return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_form(const StepParams &s, const ContractArgs &a, const void *ket, const void *bra,
                        const OutDesc &t_out, cudaStream_t st) {
  using V = typename C2T<R>::T;
  int64_t total = a.items * s.N;
  if (total <= 0) return cudaSuccess;
  form_kernel<R><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(s, a, (const V *)ket, (const V *)bra, t_out);
  tn_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_form_c(const StepParams &s, const ContractArgs &a, const float2 *ket, const float2 *bra,
                          float2 *cbuf, int64_t c_stride, cudaStream_t st) {
  const int64_t kn = s.K * s.N;
  if (kn <= 0 || a.items <= 0) return cudaSuccess;
  const int64_t tk = s.phys * s.ket_sig, tb = s.phys * s.bra_sig;   // the node's tensors
  // staged only when both operands are node tensors of that size (a double-layer step's own
  // tensor has physical stride 0 and is read in place)
  if (s.ket_sig > 0 && s.bra_sig > 0 && (tk + tb) * (int64_t)sizeof(float2) <= 48 * 1024 && kn >= 1024) {
    const int64_t gx = (kn + 256 * FORM_E - 1) / (256 * FORM_E);
    for (int64_t i0 = 0; i0 < a.items; i0 += 65535) {
      const int64_t ni = a.items - i0 < 65535 ? a.items - i0 : 65535;
      form_c_smem_kernel<<<dim3((unsigned)gx, (unsigned)ni), 256, (size_t)(tk + tb) * sizeof(float2), st>>>(
          s, a, ket, bra, cbuf, c_stride, tk, tb, i0);
    }
    tn_count_launch(1);
    return cudaGetLastError();
  }
  for (int64_t i0 = 0; i0 < a.items; i0 += 65535) {
    const int64_t ni = a.items - i0 < 65535 ? a.items - i0 : 65535;
    form_c_kernel<<<dim3((unsigned)((kn + 255) / 256), (unsigned)ni), 256, 0, st>>>(s, a, ket, bra, cbuf, c_stride,
                                                                                  i0);
  }
  tn_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_form_b_pieces(const StepParams &s, const ContractArgs &a, const float2 *ket, const float2 *bra,
                                 const Pieces &B, cudaStream_t st) {
  const int64_t kn = s.K * s.N;
  if (kn <= 0 || a.items <= 0) return cudaSuccess;
  for (int64_t i0 = 0; i0 < a.items; i0 += 65535) {
    const int64_t ni = a.items - i0 < 65535 ? a.items - i0 : 65535;
    form_b_kernel<<<dim3((unsigned)((kn + 255) / 256), (unsigned)ni), 256, 0, st>>>(s, a, ket, bra, B, i0);
  }
  tn_count_launch(1);
  return cudaGetLastError();
}

// (K, N) pairs with a compile-time streaming kernel
#define TN_FIXED_LIST(X) \
  X(4, 4) X(1, 4) X(4, 1) X(2, 2) X(2, 4) X(4, 2) X(1, 2) X(2, 1) X(4, 16) X(16, 4) X(16, 1) X(1, 16) \
  X(8, 8) X(8, 4) X(4, 8) X(8, 2) X(2, 8) X(16, 16) X(16, 8) X(8, 16)

// complex128 keeps to K * N <= 32: a larger C tile held in registers spills
template <typename R> constexpr bool fixed_fits(int k, int n) { return sizeof(R) == 4 || k * n <= 32; }

static bool has_fixed(int64_t K, int64_t N, bool fp64) {
#define TN_HAS(k, n) if (K == k && N == n) return fp64 ? fixed_fits<double>(k, n) : fixed_fits<float>(k, n);
  TN_FIXED_LIST(TN_HAS)
#undef TN_HAS
  return false;
}

bool simt_variant_ok(const StepParams &s, int v, bool fp64) {
  switch (v) {
    case SIMT_AUTO: case SIMT_T64: case SIMT_T128: case SIMT_T256: return true;
    case SIMT_STREAM: return s.K <= 16 && s.N <= 16;
    case SIMT_FIXED: return has_fixed(s.K, s.N, fp64);
    case SIMT_SMALL: return s.M * s.N <= 256;
    case SIMT_NARROW: return s.M <= 16 && s.M * s.K <= 2048;
    case SIMT_BOX: return s.box_tm > 0 && s.K * s.N <= TN_BOX_MAXKN && s.N <= TN_BOX_MAXN;
    default: return false;
  }
}

template <typename R>
cudaError_t launch_step(const StepParams &s, const ContractArgs &a, const void *ket, const void *bra,
                        const void *t_in, const OutDesc &t_out, cudaStream_t st, int variant) {
  using V = typename C2T<R>::T;
  if (a.items <= 0) return cudaSuccess;
  if (!simt_variant_ok(s, variant, sizeof(R) == 8)) return cudaErrorInvalidValue;
  if (variant == SIMT_AUTO) {   // the shape heuristic
    if (s.M >= 512 && has_fixed(s.K, s.N, sizeof(R) == 8)) variant = SIMT_FIXED;
    else if (s.K <= 16 && s.N <= 16 && s.M >= 512) variant = SIMT_STREAM;
    else if (s.M * s.N <= 16) variant = SIMT_SMALL;
    else if (s.M <= 16 && s.M * s.K <= 2048 && s.N >= 256) variant = SIMT_NARROW;
    else variant = s.N >= 48 ? SIMT_T64 : s.N >= 12 ? SIMT_T128 : SIMT_T256;
  }
  switch (variant) {
    case SIMT_BOX: return launch_step_box<R>(s, a, ket, bra, t_in, t_out, st);
    case SIMT_FIXED:
#define TN_FIXED(k, n)                                                                   \
  if (s.K == k && s.N == n) {                                                            \
    if constexpr (fixed_fits<R>(k, n)) return launch_stream_fixed<R, k, n>(s, a, ket, bra, t_in, t_out, st); \
    return cudaErrorInvalidValue;                                                        \
  }
      TN_FIXED_LIST(TN_FIXED)
#undef TN_FIXED
      return cudaErrorInvalidValue;
    case SIMT_STREAM: {
      const int64_t rows = 1024;
      const int64_t grid = ((s.M + rows - 1) / rows) * a.items;
      if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
      step_stream_kernel<R><<<(unsigned)grid, 256, 0, st>>>(s, a, (const V *)ket, (const V *)bra, (const V *)t_in,
                                                            t_out, rows);
      tn_count_launch(1);
      return cudaGetLastError();
    }
    case SIMT_NARROW: {
      const int64_t grid = ((s.N + 255) / 256) * a.items;
      if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
      step_narrow_kernel<R><<<(unsigned)grid, 256, 0, st>>>(s, a, (const V *)ket, (const V *)bra, (const V *)t_in,
                                                            t_out);
      tn_count_launch(1);
      return cudaGetLastError();
    }
    case SIMT_SMALL: {
      if (a.items > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
      const size_t node_bytes = (size_t)(s.phys * s.ket_sig + s.phys * s.bra_sig) * sizeof(V);
      const int staged = (s.ket_sig > 0 && s.bra_sig > 0 && node_bytes <= 32 * 1024) ? 1 : 0;
      step_small_kernel<R><<<(unsigned)a.items, 256, staged ? node_bytes : 0, st>>>(
          s, a, (const V *)ket, (const V *)bra, (const V *)t_in, t_out, staged);
      tn_count_launch(1);
      return cudaGetLastError();
    }
    case SIMT_T64: return launch_tiled<R, 64, 64, 8, 4, 4>(s, a, ket, bra, t_in, t_out, st);
    case SIMT_T128: return launch_tiled<R, 128, 16, 8, 8, 2>(s, a, ket, bra, t_in, t_out, st);
    default: return launch_tiled<R, 256, 4, 8, 8, 1>(s, a, ket, bra, t_in, t_out, st);
  }
}

template <typename R>
cudaError_t launch_slice_sum(const void *res, int64_t items_stride, int64_t n_bits, int64_t n_slices,
                             int accumulate, double2 *out, cudaStream_t st) {
  using V = typename C2T<R>::T;
  if (n_bits <= 0) return cudaSuccess;
  slice_sum_kernel<R><<<(unsigned)((n_bits + 255) / 256), 256, 0, st>>>((const V *)res, items_stride, n_bits,
                                                                        n_slices, accumulate, out);
  tn_count_launch(1);
  return cudaGetLastError();
}

template cudaError_t launch_form<double>(const StepParams &, const ContractArgs &, const void *, const void *,
                                         const OutDesc &, cudaStream_t);
template cudaError_t launch_form<float>(const StepParams &, const ContractArgs &, const void *, const void *,
                                        const OutDesc &, cudaStream_t);
template cudaError_t launch_step<double>(const StepParams &, const ContractArgs &, const void *, const void *,
                                         const void *, const OutDesc &, cudaStream_t, int);
template cudaError_t launch_step<float>(const StepParams &, const ContractArgs &, const void *, const void *,
                                        const void *, const OutDesc &, cudaStream_t, int);
template cudaError_t launch_slice_sum<double>(const void *, int64_t, int64_t, int64_t, int, double2 *, cudaStream_t);
template cudaError_t launch_slice_sum<float>(const void *, int64_t, int64_t, int64_t, int, double2 *, cudaStream_t);

// Box-tiled streaming contraction step (SIMT complex FMA) for thin steps: small K and N, many
// rows, the shape of every step of the double-layer network (ket and bra tensors absorbed one at
// a time, the sums of Eq. overlap without the per-qubit overlap tensors) and of the thin steps
// of the overlap network.
//
// One step computes, per (bitstring, slice) item, T_out[orow(m) + ocol(n)] = sum_k T_in[m][k]
// C[k][n] with C[k][n] the absorbed node's operand (Eq. overlap; for a double-layer step one
// tensor against the unit operand). Such a step moves 8 (M K + M N) bytes per item for 8 M K N
// flops, at most about 1.6 flops per byte here, so HBM bandwidth bounds it. The kernel is laid
// out for that roof:
//  * a CTA works on one item: it builds C in shared memory once, then walks row tiles of box_tm
//    rows whose input is one contiguous block of box_tm * K complex values, copied with 16-byte
//    cp.async into one of two buffers while the previous tile is computed and written;
//  * each thread computes two rows' group of TN consecutive columns from shared memory;
//  * the tile's outputs go out in increasing output offset (a table the plan compiler sorts: per
//    output its place in the tile and its offset), so that the permuted layout of the next step is
//    written with full, coalesced sectors; outputs adjacent both in the tile and in the next
//    layout move as one 16-byte value.
#include <cuda_runtime.h>

#include "tn_device.h"
#include "tn_internal.h"

namespace {

template <typename R> struct BoxT;
template <> struct BoxT<double> { using V = double2; };
template <> struct BoxT<float> { using V = float2; };

__device__ __forceinline__ void cp_async16(void *smem, const void *g) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *g) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Shared memory of one CTA: C[K][N], two input tile buffers [tm][kp] (the next tile is copied in
// while the current one is used) and the output tile [tm][np] (rows padded against bank
// conflicts; np is even for complex64, so an even column starts a 16-byte pair).
struct BoxLayout {
  int kp, np;
  size_t c_off, in_off, in_size, out_off, bytes;
};

__host__ __device__ inline size_t box_align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename V>
__host__ __device__ inline BoxLayout box_layout(int tm, int K, int N) {
  BoxLayout L;
  if (sizeof(V) == 8) {           // complex64: 16-byte row chunks when K is even
    L.kp = (K % 2 == 0) ? (K >= 8 ? K + 2 : K) : K;
    L.np = (N % 2 == 0) ? N + 2 : N + 1;
  } else {                        // complex128: one element per 16-byte copy
    L.kp = (K % 2 == 0) ? K + 1 : K;
    L.np = (N % 2 == 0) ? N + 1 : N;
  }
  L.c_off = 0;
  L.in_off = box_align16(L.c_off + (size_t)K * N * sizeof(V));
  L.in_size = box_align16((size_t)tm * L.kp * sizeof(V));      // one of the two input tile buffers
  L.out_off = L.in_off + 2 * L.in_size;
  L.bytes = box_align16(L.out_off + (size_t)tm * L.np * sizeof(V));
  return L;
}

// TN consecutive entries of one row of C (TN = 4 or 2 complex64: 16-byte loads)
template <int TN, typename V>
__device__ __forceinline__ void load_c(const V *p, V c[TN]) {
  if constexpr (sizeof(V) == 8 && TN % 2 == 0) {
#pragma unroll
    for (int j = 0; j < TN; j += 2) {
      const float4 q = *reinterpret_cast<const float4 *>(p + j);
      c[j].x = q.x;
      c[j].y = q.y;
      c[j + 1].x = q.z;
      c[j + 1].y = q.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < TN; ++j) c[j] = p[j];
  }
}

template <typename R, int TN>
__global__ void __launch_bounds__(256)
step_box_kernel(StepParams s, ContractArgs a, const typename BoxT<R>::V *ket, const typename BoxT<R>::V *bra,
                const typename BoxT<R>::V *tin, OutDesc out, int64_t tpc) {
  using V = typename BoxT<R>::V;
  extern __shared__ __align__(16) unsigned char box_raw[];
  const int TM = s.box_tm, K = (int)s.K, N = (int)s.N;
  const BoxLayout L = box_layout<V>(TM, K, N);
  V *Cs = reinterpret_cast<V *>(box_raw + L.c_off);
  V *const Ins0 = reinterpret_cast<V *>(box_raw + L.in_off);
  V *const Ins1 = reinterpret_cast<V *>(box_raw + L.in_off + L.in_size);
  V *Outs = reinterpret_cast<V *>(box_raw + L.out_off);
  const int tid = threadIdx.x;
  const int64_t T = s.M / TM;                    // row tiles per item
  const int64_t cpi = (T + tpc - 1) / tpc;       // CTAs per item
  const int64_t item = (int64_t)blockIdx.x / cpi;
  const int64_t t_begin = ((int64_t)blockIdx.x % cpi) * tpc;
  const int64_t t_end = t_begin + tpc < T ? t_begin + tpc : T;
  const ItemCtx c = item_ctx(a, s, item);
  const V *tp = tin + item * a.t_stride;
  const bool k_pow2 = (K & (K - 1)) == 0;
  const int k_log = __ffs(K) - 1;

  // the input tile t: box_tm rows of K values, contiguous at t * box_tm * K, into buffer t & 1
  auto load = [&](int64_t t) {
    const V *src = tp + t * (int64_t)TM * K;
    V *const Ins = (t & 1) ? Ins1 : Ins0;
    if (sizeof(V) == 8 && K % 2 == 0) {
      const int n2 = TM * K / 2, kh = K / 2;
      for (int e = tid; e < n2; e += 256) {
        const int r = k_pow2 ? (e >> (k_log - 1)) : e / kh;
        cp_async16(Ins + r * L.kp + 2 * (e - r * kh), src + 2 * e);
      }
    } else {
      for (int e = tid; e < TM * K; e += 256) {
        const int r = k_pow2 ? (e >> k_log) : e / K;
        if (sizeof(V) == 8) cp_async8(Ins + r * L.kp + (e - r * K), src + e);
        else cp_async16(Ins + r * L.kp + (e - r * K), src + e);
      }
    }
    cp_async_commit();
  };
  if (t_begin < t_end) load(t_begin);

  {   // the absorbed node's operand (Eq. overlap), once per CTA
    const V *kp = ket + s.ket_off + c.sa;
    const V *bp = bra + c.b * a.bra_stride + s.bra_off + c.sb;
    const int32_t *bka = a.tab + s.t_bka, *bkb = a.tab + s.t_bkb;
    const int32_t *bna = a.tab + s.t_bna, *bnb = a.tab + s.t_bnb;
    for (int i = tid; i < K * N; i += 256) {
      const int k = i / N, n = i - k * N;
      Cs[i] = overlap_elem(kp, bp, (int64_t)bka[k] + bna[n], (int64_t)bkb[k] + bnb[n], s.ket_sig, s.bra_sig, s.phys);
    }
  }

  const int G = N / TN;                 // threads per row
  const int RP = 256 / G;               // rows per pass
  const int g = tid % G, r0 = tid / G;
  const int2 *wtab = reinterpret_cast<const int2 *>(a.tab + s.t_wperm);   // (r << 16 | n, offset) per output
  for (int64_t t = t_begin; t < t_end; ++t) {
    // the next tile's copy runs while this tile is computed and written (its buffer was last read
    // by the compute of tile t - 1, which every thread finished before the barrier below it)
    if (t + 1 < t_end) {
      load(t + 1);
      cp_async_wait_one();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();                    // input tile t and C in place; the last tile's outputs written
    const V *const Ins = (t & 1) ? Ins1 : Ins0;
    if (r0 < RP) {
      // two rows per pass (r and r + RP) against the same C entries
      for (int r = r0; r < TM; r += 2 * RP) {
        const bool two = r + RP < TM;
        V acc0[TN], acc1[TN];
#pragma unroll
        for (int j = 0; j < TN; ++j) acc0[j] = acc1[j] = cz<V>();
        const V *xr0 = Ins + r * L.kp;
        const V *xr1 = two ? xr0 + RP * L.kp : xr0;
        const V *cc = Cs + g * TN;
#pragma unroll 4
        for (int k = 0; k < K; ++k) {
          const V x0 = xr0[k], x1 = xr1[k];
          V cv[TN];
          load_c<TN>(cc + k * N, cv);
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            acc0[j] = cfma(x0, cv[j], acc0[j]);
            acc1[j] = cfma(x1, cv[j], acc1[j]);
          }
        }
        V *o = Outs + r * L.np + g * TN;
#pragma unroll
        for (int j = 0; j < TN; ++j) o[j] = acc0[j];
        if (two) {
          o += RP * L.np;
#pragma unroll
          for (int j = 0; j < TN; ++j) o[j] = acc1[j];
        }
      }
    }
    __syncthreads();                    // output tile complete
    const int obase = orow_of(s, t * (int64_t)TM);
    const int tot = TM * N;
    for (int e = 2 * tid; e < tot; e += 512) {
      const int2 w0 = __ldg(wtab + e);
      const V *src0 = Outs + ((w0.x >> 16) & 0x3fff) * L.np + (w0.x & 0xffff);
      if constexpr (sizeof(V) == 8) {
        // a marked pair (same row, columns n, n + 1, offsets d, d + 1, n and d even): one 16-byte
        // move when the tile's output base keeps it aligned
        if (((w0.x >> 30) & 1) && out.fmt == 0 && ((obase + w0.y) & 1) == 0) {
          float2 *dst = reinterpret_cast<float2 *>(out.p) + item * a.t_stride + obase + w0.y;
          *reinterpret_cast<float4 *>(dst) = *reinterpret_cast<const float4 *>(src0);
          continue;
        }
      }
      store_out(out, a.t_stride, item, obase + w0.y, *src0);
      if (e + 1 < tot) {
        const int2 w1 = __ldg(wtab + e + 1);
        store_out(out, a.t_stride, item, obase + w1.y, Outs[((w1.x >> 16) & 0x3fff) * L.np + (w1.x & 0xffff)]);
      }
    }
  }
}

template <typename R, int TN>
cudaError_t launch_tn(const StepParams &s, const ContractArgs &a, const void *ket, const void *bra, const void *t_in,
                      const OutDesc &out, cudaStream_t st) {
  using V = typename BoxT<R>::V;
  const BoxLayout L = box_layout<V>(s.box_tm, (int)s.K, (int)s.N);
  if (L.bytes > 48 * 1024) {
    const int lim = tn_smem_optin<step_box_kernel<R, TN>>();
    if (lim < 0 || (size_t)lim < L.bytes) return cudaErrorInvalidValue;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // tiles per CTA: whole items when there are enough of them to fill every SM many times over,
  // else the items' tiles spread over more CTAs
  const int64_t T = s.M / s.box_tm;
  int64_t tpc = T * a.items / ((int64_t)sms * 16);
  tpc = tpc < 1 ? 1 : tpc > T ? T : tpc;
  const int64_t cpi = (T + tpc - 1) / tpc;
  const int64_t grid = cpi * a.items;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  step_box_kernel<R, TN><<<(unsigned)grid, 256, L.bytes, st>>>(s, a, (const V *)ket, (const V *)bra, (const V *)t_in,
                                                               out, tpc);
  tn_count_launch(1);
  return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_step_box(const StepParams &s, const ContractArgs &a, const void *ket, const void *bra,
                            const void *t_in, const OutDesc &out, cudaStream_t st) {
  if (a.items <= 0) return cudaSuccess;
  if (s.box_tm <= 0 || s.M % s.box_tm != 0 || s.K * s.N > TN_BOX_MAXKN || s.N > TN_BOX_MAXN)
    return cudaErrorInvalidValue;
  if (s.N % 4 == 0) return launch_tn<R, 4>(s, a, ket, bra, t_in, out, st);
  if (s.N % 2 == 0) return launch_tn<R, 2>(s, a, ket, bra, t_in, out, st);
  return launch_tn<R, 1>(s, a, ket, bra, t_in, out, st);
}

template cudaError_t launch_step_box<double>(const StepParams &, const ContractArgs &, const void *, const void *,
                                             const void *, const OutDesc &, cudaStream_t);
template cudaError_t launch_step_box<float>(const StepParams &, const ContractArgs &, const void *, const void *,
                                            const void *, const OutDesc &, cudaStream_t);

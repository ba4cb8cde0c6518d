// Step-kernel autotuner.
//
// Every contraction step of a plan (one TTGT pairwise contraction of the path) can run on several
// kernels: SIMT tiles of three shapes, two streaming kernels for small K and N, a one-CTA-per-item
// reduction for tiny outputs, and, for the tensor-core forms, the tcgen05 kernel with in-kernel
// operand split or the TMA-fed tcgen05 kernel (BF16x6) with 128- or 64-column tiles, its overlap
// operand built on chip from the node tensors, formed in HBM as complex64 and split on chip, or
// formed in HBM as bf16 pieces and loaded. The shape
// heuristic picks one; the autotuner times every kernel that supports the step on the plan's own
// workspace, at the batch size given, and keeps the fastest. Most TMA-fed kernels read their input
// as bf16 pieces, which the previous step then has to write: each candidate is charged the
// previous step's time in the output format it implies; a second pass then re-picks each step's kernel in
// its final output format. The heuristic's kernel is kept unless another is at least 3% faster. Choices are stored in the plan per precision and used by every
// later tn_amplitudes, tn_amplitudes_static, server and batch call on that plan. A workspace the
// tuner had to allocate is released before it returns.
#include <algorithm>
#include <cstring>

#include "tn_host.h"

namespace {

const int kCandidates[] = {SIMT_AUTO, SIMT_T64,  SIMT_T128, SIMT_T256, SIMT_STREAM, SIMT_FIXED, SIMT_SMALL, SIMT_NARROW, SIMT_BOX, SK_TC,
                           SK_TMA,    SK_TMA128, SK_TMA64,  SK_TMAF,   SK_TMAF128,  SK_TMAF64,  SK_TMAC,    SK_TMAC128,
                           SK_TMAC64, SK_TMAP,   SK_TMAP128, SK_TMAP64,  SK_TMAPA,    SK_TMAPA128, SK_TMAPA64,
                           SK_TMAPF,  SK_TMAPF128, SK_TMAPF64, SK_TMAPFA, SK_TMAPFA128, SK_TMAPFA64};

struct Events {
  cudaEvent_t a = nullptr, b = nullptr;
  Events() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Events() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

}  // namespace

extern "C" tn_status tn_autotune(tn_plan *p, tn_precision prec, int64_t n_bits, void *cuda_stream, int32_t *kernels) {
  if (!p) return tn_fail(TN_ERR_ARG, "tn_autotune: NULL plan");
  if (prec < TN_FP64 || prec > TN_TF32X6) return tn_fail(TN_ERR_ARG, "unknown precision %d", (int)prec);
  if (n_bits < 0) return tn_fail(TN_ERR_ARG, "tn_autotune: negative batch size");
  tn_circuit *c = p->c;
  if (p->generation != c->generation) return tn_fail(TN_ERR_STATE, "plan is stale: the circuit was re-evolved");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int kind = prec == TN_FP64 ? 0 : 1;
  Workspace &w = p->ws;
  const bool had_ws = w.t0.p != nullptr;   // a workspace made here is released again at the end
  const int64_t want = n_bits > 0 ? std::min<int64_t>(std::max<int64_t>(n_bits, w.chunk), p->chunk[kind]) : p->chunk[kind];
  tn_status s = ws_ensure_sized(p, w, kind, want, p->slice_chunk[kind], st);
  if (s != TN_OK) return s;
  const int64_t nb = n_bits > 0 ? std::min<int64_t>(n_bits, w.chunk) : w.chunk;
  const int words = (c->n + 63) / 64;
  p->tune[prec].clear();
  std::vector<int> ks = step_kernels(p, prec);
  // one full pass with the heuristic kernels on the all-zero bitstring: fills the bra tensors and
  // every buffer the steps read (their timing does not depend on the values)
  CUDA_TRY(cudaMemsetAsync(w.bits.p, 0, (size_t)nb * words * 8, st));
  CUDA_TRY(cudaMemsetAsync(w.err.p, 0, 2 * sizeof(int), st));
  CUDA_TRY(cudaMemsetAsync(w.t0.p, 0, w.t0.bytes, st));
  CUDA_TRY(cudaMemsetAsync(w.t1.p, 0, w.t1.bytes, st));
  if (w.cbuf.p) CUDA_TRY(cudaMemsetAsync(w.cbuf.p, 0, w.cbuf.bytes, st));
  s = enqueue_chunk(p, w, (const uint64_t *)w.bits.p, nb, prec, ks, (double2 *)w.res.p, st);
  if (s != TN_OK) return s;
  int err[2] = {0, 0};
  CUDA_TRY(cudaMemcpyAsync(err, w.err.p, sizeof err, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if ((s = check_err_words(err)) != TN_OK) return s;

  const int64_t sg = std::min<int64_t>(w.slice_chunk, p->n_slices);
  ContractArgs a;
  a.tab = (const int32_t *)p->tab_dev.p;
  a.n_slices = sg;
  a.slice0 = 0;
  a.items = nb * sg;
  a.t_stride = p->maxT;
  a.bra_stride = p->net.bra_elems;
  const void *ket = p->net.merged() ? (kind ? w.ket32.p : w.ket64.p) : (kind ? c->ket_c64.p : c->ket_dev.p);
  const void *bra = kind ? w.bra32.p : w.bra64.p;
  const int64_t cap = (int64_t)w.chunk * w.slice_chunk;
  Events ev;
  if (!ev.a || !ev.b) return tn_fail(TN_ERR_CUDA, "tn_autotune: cudaEventCreate failed");
  // one step's launch time with kernel k, writing its output in format fmt (0 complex64, 1 the
  // bf16 pieces a TMA-fed consumer reads): one untimed launch, then enough for about 0.5 ms
  auto time_of = [&](size_t j, int k, int fmt, float &ms) -> tn_status {
    OutDesc od;
    od.p = w.t1.p;
    od.fmt = fmt;
    od.plane_u32 = cap * p->maxT;
    ms = 0;
    cudaError_t e = cudaSuccess;
    for (int rep = 0, r = 1; rep < 2; ++rep) {
      CUDA_TRY(cudaEventRecord(ev.a, st));
      const void *kj, *bj;
      ContractArgs aj;
      step_operands(p, j, kind, ket, bra, a, kj, bj, aj);
      for (int i = 0; i < r && e == cudaSuccess; ++i)
        e = enqueue_step(p, w, j, k, prec, aj, kj, bj, w.t0.p, w.t1.p, od, st);
      if (e != cudaSuccess) {
        cudaStreamSynchronize(st);
        return tn_fail(TN_ERR_CUDA, "step %zu kernel %d: %s", j, k, cudaGetErrorString(e));
      }
      CUDA_TRY(cudaEventRecord(ev.b, st));
      CUDA_TRY(cudaEventSynchronize(ev.b));
      float t = 0;
      CUDA_TRY(cudaEventElapsedTime(&t, ev.a, ev.b));
      ms = t / (float)r;
      r = std::max(1, std::min(50, (int)(0.5f / std::max(ms, 1e-4f))));
    }
    return TN_OK;
  };
  for (size_t j = 1; j < p->steps.size(); ++j) {
    const StepParams &sp = p->steps[j];
    const int fmt = (j + 1 < ks.size() && sk_reads_pieces(ks[j + 1])) ? 1 : 0;
    // a kernel here that reads bf16 pieces makes the previous step write them: each candidate is
    // charged the previous step's time (its chosen kernel) in the output format it implies
    float prev_ms[2] = {0, 0};
    if (j >= 2 && prec == TN_BF16X6) {
      for (int f = 0; f < 2; ++f) {
        tn_status ts = time_of(j - 1, ks[j - 1], f, prev_ms[f]);
        if (ts != TN_OK) return ts;
      }
    }
    const int dflt = ks[j];
    float best_ms = 0;
    tn_status ts = time_of(j, dflt, fmt, best_ms);
    if (ts != TN_OK) return ts;
    best_ms += prev_ms[sk_reads_pieces(dflt) ? 1 : 0];
    int best = dflt;
    for (int k : kCandidates) {
      if (k == dflt || !step_kernel_ok(sp, prec, k)) continue;
      float ms = 0;
      ts = time_of(j, k, fmt, ms);
      if (ts != TN_OK) return ts;
      ms += prev_ms[sk_reads_pieces(k) ? 1 : 0];
      if (ms < 0.97f * best_ms) {
        best_ms = ms;
        best = k;
      }
    }
    ks[j] = best;
  }
  // second pass: each step's output format is now final (it follows the next step's choice), so
  // its kernel is chosen again in that format among those that read their input in the same format
  for (size_t j = 1; j < p->steps.size() && prec == TN_BF16X6; ++j) {
    const StepParams &sp = p->steps[j];
    const int fmt = (j + 1 < ks.size() && sk_reads_pieces(ks[j + 1])) ? 1 : 0;
    const bool pieces = sk_reads_pieces(ks[j]);
    float best_ms = 0;
    tn_status ts = time_of(j, ks[j], fmt, best_ms);
    if (ts != TN_OK) return ts;
    int best = ks[j];
    for (int k : kCandidates) {
      if (k == ks[j] || sk_reads_pieces(k) != pieces || !step_kernel_ok(sp, prec, k)) continue;
      float ms = 0;
      ts = time_of(j, k, fmt, ms);
      if (ts != TN_OK) return ts;
      if (ms < 0.97f * best_ms) {
        best_ms = ms;
        best = k;
      }
    }
    ks[j] = best;
  }
  // the bounded waits of the tensor-core kernels may have expired in any timed launch
  CUDA_TRY(cudaMemcpyAsync(err, w.err.p, sizeof err, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if ((s = check_err_words(err)) != TN_OK) return s;
  p->tune[prec] = ks;
  if (kernels)
    for (size_t j = 1; j < ks.size(); ++j) kernels[j - 1] = ks[j];
  if (!had_ws) ws_release(c->mem, w);
  return TN_OK;
}

extern "C" tn_status tn_plan_kernels(const tn_plan *p, tn_precision prec, int32_t *kernels) {
  if (!p || !kernels) return tn_fail(TN_ERR_ARG, "tn_plan_kernels: NULL argument");
  if (prec < TN_FP64 || prec > TN_TF32X6) return tn_fail(TN_ERR_ARG, "unknown precision %d", (int)prec);
  const std::vector<int> ks = step_kernels(p, prec);
  for (size_t j = 1; j < ks.size(); ++j) kernels[j - 1] = ks[j];
  return TN_OK;
}

extern "C" tn_status tn_plan_set_kernels(tn_plan *p, tn_precision prec, const int32_t *kernels) {
  if (!p) return tn_fail(TN_ERR_ARG, "tn_plan_set_kernels: NULL plan");
  if (prec < TN_FP64 || prec > TN_TF32X6) return tn_fail(TN_ERR_ARG, "unknown precision %d", (int)prec);
  if (!kernels) {
    p->tune[prec].clear();
    return TN_OK;
  }
  std::vector<int> ks(p->steps.size(), SIMT_AUTO);
  for (size_t j = 1; j < ks.size(); ++j) {
    ks[j] = kernels[j - 1];
    if (!step_kernel_ok(p->steps[j], prec, ks[j]))
      return tn_fail(TN_ERR_ARG, "tn_plan_set_kernels: kernel %d does not support step %zu (M=%lld K=%lld N=%lld)",
                     ks[j], j, (long long)p->steps[j].M, (long long)p->steps[j].K, (long long)p->steps[j].N);
  }
  p->tune[prec] = ks;
  return TN_OK;
}

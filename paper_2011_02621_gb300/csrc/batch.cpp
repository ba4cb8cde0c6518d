// Batched circuits: the amplitudes of many circuits (each with its own graph, gates, plan and batch
// of bitstrings, shapes uneven) computed by one CUDA graph launch.
//
// tn_batch_create groups the circuits into waves whose workspaces fit the memory budget side by
// side (each circuit keeps its plan's batch size), carves every wave's workspaces from one
// resident arena that the next wave reuses, runs each circuit once on the stream (this validates
// the plans and sets the kernels up), and captures the whole batch into one CUDA graph: per wave
// a fork into one branch per circuit, each branch the circuit's full path (bra evolution with the
// batched FP64 SVD, overlap formation, the path-ordered contraction steps with the plan's tuned
// kernels, the FP64 cross-slice sum), and a join before the next wave. Branches of a wave have no
// dependencies, so the device runs those circuits concurrently and small circuits fill the SMs
// together. Graphs above TN_BATCH_MAX_NODES kernel nodes are refused (a budget too small for the
// circuits' batch sizes would otherwise make one from very many tiny chunks). tn_batch_run is one
// cudaGraphLaunch.
#include <algorithm>
#include <cstring>
#include <vector>

#include "tn_host.h"

#define TN_BATCH_MAX_NODES 100000

struct tn_batch {
  struct Item {
    tn_plan *p = nullptr;
    int64_t generation = 0;
    int64_t n = 0;
    int words = 1;
    int64_t bits_off = 0, res_off = 0;   // in words / in amplitudes
    int wave = 0;
    Workspace w;                         // carved from the arena (not owned)
  };
  std::vector<Item> items;
  int n_waves = 0;
  tn_precision prec = TN_FP64;
  DevMem *mem = nullptr;                 // allocator of the shared buffers (the first plan's circuit)
  Buf bits, res, arena, errs;            // errs: two error words per circuit, outside the arena
  int64_t total_words = 0, total_amps = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_kernels = 0;
  int64_t device_bytes = 0;
};

namespace {

void destroy(tn_batch *b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->mem) {
    b->mem->release(b->bits);
    b->mem->release(b->res);
    b->mem->release(b->arena);
    b->mem->release(b->errs);
  }
  delete b;
}

// every branch's work: zero its error words, then its chunks of bitstrings
tn_status enqueue_item(tn_batch *b, tn_batch::Item &it, cudaStream_t st) {
  CUDA_TRY(cudaMemsetAsync(it.w.err.p, 0, 2 * sizeof(int), st));
  const std::vector<int> ks = step_kernels(it.p, b->prec);
  for (int64_t start = 0; start < it.n; start += it.w.chunk) {
    const int64_t nb = std::min<int64_t>(it.w.chunk, it.n - start);
    tn_status s = enqueue_chunk(it.p, it.w, (const uint64_t *)b->bits.p + it.bits_off + start * it.words, nb, b->prec,
                                ks, (double2 *)b->res.p + it.res_off + start, st);
    if (s != TN_OK) return s;
  }
  return TN_OK;
}

tn_status read_errors(tn_batch *b, cudaStream_t st) {
  std::vector<int> err(2 * b->items.size(), 0);
  for (size_t i = 0; i < b->items.size(); ++i)
    CUDA_TRY(cudaMemcpyAsync(&err[2 * i], b->items[i].w.err.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  for (size_t i = 0; i < b->items.size(); ++i) {
    tn_status s = check_err_words(&err[2 * i]);
    if (s != TN_OK) return tn_fail(s, "batch circuit %zu: %s", i, tn_last_error());
  }
  return TN_OK;
}

tn_status capture(tn_batch *b) {
  const size_t n = b->items.size();
  cudaStream_t cs = nullptr;
  std::vector<cudaStream_t> bs(n, nullptr);
  std::vector<cudaEvent_t> ev(n + 1, nullptr);
  tn_status s = TN_OK;
  auto cleanup = [&]() {
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
    for (auto x : bs)
      if (x) cudaStreamDestroy(x);
    if (cs) cudaStreamDestroy(cs);
  };
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  for (size_t i = 0; i < n && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&bs[i], cudaStreamNonBlocking);
  for (size_t i = 0; i <= n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cleanup();
    return tn_fail(TN_ERR_CUDA, "batch capture set-up: %s", cudaGetErrorString(e));
  }
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cleanup();
    return tn_fail(TN_ERR_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
  }
  const int64_t counted = tn_launch_count(0);   // captured launches run later, counted per graph launch
  e = cudaEventRecord(ev[n], cs);   // fork of the first wave
  for (int wv = 0; wv < b->n_waves && e == cudaSuccess && s == TN_OK; ++wv) {
    std::vector<size_t> members;
    for (size_t i = 0; i < n; ++i)
      if (b->items[i].wave == wv) members.push_back(i);
    for (size_t i : members) {
      if (e != cudaSuccess || s != TN_OK) break;
      e = cudaStreamWaitEvent(bs[i], ev[n], 0);
      if (e == cudaSuccess) s = enqueue_item(b, b->items[i], bs[i]);
      if (e == cudaSuccess && s == TN_OK) e = cudaEventRecord(ev[i], bs[i]);
      if (e == cudaSuccess && s == TN_OK) e = cudaStreamWaitEvent(cs, ev[i], 0);   // join
    }
    if (e == cudaSuccess && s == TN_OK) e = cudaEventRecord(ev[n], cs);   // fork of the next wave
    if (s == TN_OK && tn_launch_count(0) - counted > TN_BATCH_MAX_NODES)
      s = tn_fail(TN_ERR_UNSUPPORTED,
                  "tn_batch_create: more than %d kernels in one graph; give the batch more memory "
                  "(hbm_budget_bytes) or plans with larger batches",
                  TN_BATCH_MAX_NODES);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(cs, &g);
  tn_count_launch(counted - tn_launch_count(0));
  if (s == TN_OK && (e != cudaSuccess || ee != cudaSuccess))
    s = tn_fail(TN_ERR_CUDA, "batch capture: %s", cudaGetErrorString(e != cudaSuccess ? e : ee));
  cudaGetLastError();
  if (s != TN_OK) {
    if (g) cudaGraphDestroy(g);
    cleanup();
    return s;
  }
  b->graph = g;
  e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) {
    cleanup();
    return tn_fail(TN_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  size_t nodes = 0;
  cudaGraphGetNodes(g, nullptr, &nodes);
  std::vector<cudaGraphNode_t> all(nodes);
  if (nodes) cudaGraphGetNodes(g, all.data(), &nodes);
  b->graph_kernels = 0;
  for (auto nd : all) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) b->graph_kernels++;
  }
  cleanup();
  return TN_OK;
}

tn_status upload_bits(tn_batch *b, const uint64_t *bits, cudaStream_t st) {
  CUDA_TRY(cudaMemcpyAsync(b->bits.p, bits, (size_t)b->total_words * 8,
                           is_device_ptr(bits) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  return TN_OK;
}

}  // namespace

extern "C" tn_status tn_batch_create(tn_plan *const *plans, int32_t n_plans, const uint64_t *bits,
                                     const int64_t *n_bits, tn_precision prec, double hbm_budget_bytes,
                                     void *cuda_stream, tn_batch **out) {
  if (!out) return tn_fail(TN_ERR_ARG, "tn_batch_create: out is NULL");
  *out = nullptr;
  if (!plans || n_plans <= 0 || !bits || !n_bits) return tn_fail(TN_ERR_ARG, "tn_batch_create: bad arguments");
  if (prec < TN_FP64 || prec > TN_TF32X6) return tn_fail(TN_ERR_ARG, "unknown precision %d", (int)prec);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int kind = prec == TN_FP64 ? 0 : 1;
  tn_batch *b = new tn_batch();
  b->prec = prec;
  for (int32_t i = 0; i < n_plans; ++i) {
    tn_plan *p = plans[i];
    if (!p || n_bits[i] <= 0) {
      destroy(b);
      return tn_fail(TN_ERR_ARG, "tn_batch_create: circuit %d has no plan or no bitstrings", i);
    }
    if (p->generation != p->c->generation) {
      destroy(b);
      return tn_fail(TN_ERR_STATE, "tn_batch_create: plan %d is stale (its circuit was re-evolved)", i);
    }
    tn_batch::Item it;
    it.p = p;
    it.generation = p->generation;
    it.n = n_bits[i];
    it.words = (p->c->n + 63) / 64;
    it.bits_off = b->total_words;
    it.res_off = b->total_amps;
    b->total_words += it.n * it.words;
    b->total_amps += it.n;
    b->items.push_back(it);
  }
  b->mem = &plans[0]->c->mem;
  tn_status s = b->mem->ensure(b->bits, (size_t)b->total_words * 8, st);
  if (s == TN_OK) s = b->mem->ensure(b->res, (size_t)b->total_amps * sizeof(tn_c128), st);
  // waves: circuits in order, each with its plan's own batch size, side by side while their
  // workspaces fit the budget (a circuit alone is always a wave); one arena for the largest wave
  std::vector<WsSizes> z(b->items.size());
  std::vector<int64_t> chunk(b->items.size());
  int64_t wave_bytes = 0, arena = 0;
  for (size_t i = 0; i < b->items.size(); ++i) {
    tn_batch::Item &it = b->items[i];
    chunk[i] = std::max<int64_t>(1, std::min<int64_t>(it.n, it.p->chunk[kind]));
    z[i] = ws_sizes(it.p, kind, chunk[i], it.p->slice_chunk[kind]);
    if (i > 0 && hbm_budget_bytes > 0 && (double)(wave_bytes + z[i].total) > hbm_budget_bytes) {
      ++b->n_waves;
      wave_bytes = 0;
    }
    it.wave = b->n_waves;
    wave_bytes += z[i].total;
    arena = std::max(arena, wave_bytes);
  }
  ++b->n_waves;
  if (s == TN_OK) s = b->mem->ensure(b->arena, (size_t)std::max<int64_t>(arena, 256), st);
  if (s == TN_OK) s = b->mem->ensure(b->errs, b->items.size() * 64, st);
  if (s == TN_OK) {
    int64_t off = 0;
    int cur = -1;
    for (size_t i = 0; i < b->items.size(); ++i) {
      tn_batch::Item &it = b->items[i];
      if (it.wave != cur) { cur = it.wave; off = 0; }
      ws_carve(it.w, static_cast<unsigned char *>(b->arena.p) + off, z[i], chunk[i], it.p->slice_chunk[kind], st);
      it.w.err.p = static_cast<unsigned char *>(b->errs.p) + i * 64;   // survives the later waves
      off += z[i].total;
    }
  }
  b->device_bytes = (int64_t)(b->bits.bytes + b->res.bytes + b->arena.bytes + b->errs.bytes);
  if (s == TN_OK) s = upload_bits(b, bits, st);
  // one eager pass: validates every plan and sets the kernels up before the capture
  for (auto &it : b->items)
    if (s == TN_OK) s = enqueue_item(b, it, st);
  if (s == TN_OK) s = read_errors(b, st);
  if (s == TN_OK) s = capture(b);
  if (s != TN_OK) {
    destroy(b);
    return s;
  }
  *out = b;
  return TN_OK;
}

extern "C" tn_status tn_batch_set_bits(tn_batch *b, const uint64_t *bits, void *cuda_stream) {
  if (!b || !bits) return tn_fail(TN_ERR_ARG, "tn_batch_set_bits: NULL argument");
  return upload_bits(b, bits, (cudaStream_t)cuda_stream);
}

extern "C" tn_status tn_batch_run(tn_batch *b, void *cuda_stream) {
  if (!b) return tn_fail(TN_ERR_ARG, "tn_batch_run: NULL batch");
  for (size_t i = 0; i < b->items.size(); ++i)
    if (b->items[i].p->c->generation != b->items[i].generation)
      return tn_fail(TN_ERR_STATE, "tn_batch_run: circuit %zu was re-evolved after the batch was made", i);
  CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)cuda_stream));
  tn_count_launch(b->graph_kernels);
  return TN_OK;
}

extern "C" tn_status tn_batch_read(tn_batch *b, tn_c128 *out, void *cuda_stream) {
  if (!b || !out) return tn_fail(TN_ERR_ARG, "tn_batch_read: NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  CUDA_TRY(cudaMemcpyAsync(out, b->res.p, (size_t)b->total_amps * sizeof(tn_c128),
                           is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  return read_errors(b, st);
}

extern "C" tn_status tn_batch_info(const tn_batch *b, int64_t *graph_kernels, int64_t *device_bytes) {
  if (!b) return tn_fail(TN_ERR_ARG, "tn_batch_info: NULL batch");
  if (graph_kernels) *graph_kernels = b->graph_kernels;
  if (device_bytes) *device_bytes = b->device_bytes;
  return TN_OK;
}

extern "C" void tn_batch_free(tn_batch *b) { destroy(b); }

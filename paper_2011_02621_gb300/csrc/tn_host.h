// Host-side structures behind the opaque handles of include/tn.h.
#pragma once

#include <array>
#include <utility>
#include <vector>

#include "tn_internal.h"

tn_status tn_fail(tn_status s, const char *fmt, ...);

struct Buf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = 0;
};

// Device memory through the caller's allocator, else cudaMalloc / cudaFree.
struct DevMem {
  tn_allocator a{};
  bool has = false;
  void *alloc(size_t bytes, cudaStream_t st);
  void release(Buf &b);
  tn_status ensure(Buf &b, size_t bytes, cudaStream_t st);
};

// One half of the two-sided evolution: the fused gate program in processing
// order with its static bond bounds and node slots.
struct Half {
  std::vector<int> dims;                          // structural bond dims after the program
  std::vector<GateParams> gp;                     // two-qubit steps
  std::vector<std::pair<int, int>> gate_nodes;    // (k, l) per two-qubit step
  std::vector<Apply1Params> ap;                   // trailing single-qubit applications
  std::vector<int> ap_node;
  std::vector<std::pair<int, int>> seq;           // (2, gp index) or (1, ap index)
  std::vector<int64_t> node_off;                  // slot offsets (complex elements)
  int64_t item_elems = 2;                         // elements per item (all slots)
  int64_t max_work = 0;                           // global SVD work per item (steps not fitting smem)
  int64_t max_gate_mn = 0;
};

struct tn_circuit {
  int n = 0, ne = 0, max_deg = 0;
  std::vector<int> eu, ev;
  std::vector<std::vector<int>> legs;             // incident edge ids, increasing
  std::vector<tn_gate> gates;
  DevMem mem;
  bool evolved = false;
  int64_t generation = 0;
  int split = 0, chi = 0;
  double cutoff = 1e-12;
  int device = 0;
  Half ket, bra;
  Buf ket_dev, ket_c64, ket_off_dev, bra_off_dev, err_dev, ket_work;
};

struct Workspace {
  int chunk = 0;
  int64_t slice_chunk = 1;
  Buf bits, bra64, bra32, gwork, t0, t1, res, err, cbuf;
};

struct tn_plan {
  tn_circuit *c = nullptr;
  int64_t generation = 0;
  std::vector<int> order, cuts;
  double score = 0;
  int64_t pops = 0;
  int rank_used = 0;
  int64_t n_slices = 1;
  std::vector<StepParams> steps;                  // steps[0] forms the first node's C tensor
  std::vector<std::array<int64_t, 3>> step_mkn;
  std::vector<int32_t> tab_host;
  Buf tab_dev;
  int64_t maxT = 1;
  int64_t maxKN = 1;                              // largest overlap tensor of a step (elements)
  double cmacs = 0, bytes = 0;
  int chunk[2] = {1, 1};                          // bitstrings per batch: [FP64, complex64]
  int64_t slice_chunk[2] = {1, 1};                // slices per launch group (all S when chunk > 1)
  int64_t ws_bytes[2] = {0, 0};
  Workspace ws;
};

tn_path_opts tn_default_opts();
int64_t plan_ws_bytes(const tn_plan *p, int kind, int64_t chunk, int64_t slices);
tn_status ws_ensure(tn_plan *p, Workspace &w, int kind, cudaStream_t st);
void ws_release(DevMem &mem, Workspace &w);
tn_status run_amplitudes(tn_plan *p, Workspace &w, const uint64_t *bits, int64_t n, tn_precision prec,
                         tn_c128 *out, cudaStream_t st);
tn_status run_half(const Half &h, int n_qubits, double2 *base, int items, const int64_t *node_off_dev,
                   const uint64_t *bits_dev, int words, double2 *gwork, int *errflag, cudaStream_t st);

// tracing: events around launches, attributed to a kernel kind
struct ProfScope {
  int slot = -1;
  cudaStream_t st = 0;
  ProfScope(const char *kind, cudaStream_t stream, double bytes, double flops);
  ~ProfScope();
};

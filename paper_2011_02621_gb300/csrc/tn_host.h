// Host-side structures behind the opaque handles of include/tn.h.
#pragma once

#include <array>
#include <utility>
#include <vector>

#include "tn_internal.h"

tn_status tn_fail(tn_status s, const char *fmt, ...);

// return TN_ERR_CUDA with the failing call's text from a function returning tn_status
#define CUDA_TRY(x)                                                                           \
  do {                                                                                        \
    cudaError_t e_ = (x);                                                                     \
    if (e_ != cudaSuccess) return tn_fail(TN_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

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
  int max_sweeps = 0;                             // Jacobi sweep cap of every SVD (0: the default)
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
  int compress = 0;                               // bond compression for the next programs (tn_compress)
  int built_compress = 0;                         // the compression of the current programs
  int device = 0;
  int max_sweeps = 0;                             // tn_set_svd_sweeps (0: the default)
  Half ket, bra;
  Buf ket_dev, ket_c64, ket_off_dev, bra_off_dev, err_dev, ket_work;
};

struct Workspace {
  int chunk = 0;
  int64_t slice_chunk = 1;
  bool fixed = false;                             // carved in memory the caller owns: never grown or freed
  Buf bits, bra64, bra32, gwork, t0, t1, res, err, cbuf;
  Buf ket64, ket32;                               // the ket with merged nodes (plans that merge)
};

// The overlap network a plan contracts: one node per qubit, or fewer when boundary nodes were
// merged into a neighbour (exactly, on both halves, before the contraction). Edge ids are the
// network's own; eid maps them to the circuit's edge ids. A node tensor is [p][legs in order],
// p its physical index (phys values), stored in the ket item (one) and in every bitstring's bra
// item at the node's offsets; merged nodes live past the halves' own slots.
struct Net {
  int n = 0, ne = 0;
  std::vector<int> eu, ev, eid;
  std::vector<std::vector<int>> legs;             // per node, network edge ids in tensor order
  std::vector<int> rep;                           // representative qubit per node
  std::vector<int> owner;                         // per qubit: the node it belongs to
  std::vector<int> phys;                          // physical values per node
  std::vector<int64_t> dk, db;                    // ket / bra dim per network edge
  std::vector<int64_t> ket_off, bra_off;          // node offsets in the ket / bra item
  int64_t ket_elems = 0, bra_elems = 0;           // item sizes including merged nodes
  std::vector<MergeParams> mk, mb;                // merge program of the ket / bra, in order
  // Double-layer networks only (empty otherwise): 1 = the node is a ket tensor, 2 = a bra tensor.
  // Such a node has one tensor, [legs in order] with leg dims dc, in its own half's item; the
  // other operand slot of its steps reads the plan's two-value unit tensor [1, 0].
  std::vector<int> layer;
  std::vector<int> dl_id;                         // double-layer nodes: the original node id (0 .. 2n-1)
  int64_t dc(int e) const { return dk[e] * db[e]; }
  bool merged() const { return !mk.empty() || !mb.empty(); }
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
  Net net;                                        // nodes, legs and layouts the steps address
  std::vector<int> step_layer;                    // per step: 0, or the absorbed node's layer (1 ket, 2 bra)
  Buf unit_dev;                                   // double-layer plans: [1, 0] as complex128, then as complex64
  std::vector<int> tune[TN_TF32X6 + 1];           // per precision: a StepKernel per step (empty: heuristic)
};

// Kernel of one contraction step: a SimtVariant (SIMT, complex FMA), tcgen05 with the operand split in
// the kernel, or TMA-fed tcgen05 (BF16x6) with a shape-picked or fixed tile width, building the
// overlap operand in shared memory (SK_TMA*), loading it after a formation pass (SK_TMAF*), or
// splitting its complex64 form on chip, one tile per CTA (SK_TMAC*) or persistent (SK_TMAP*).
enum StepKernel {
  SK_TC = 16,
  SK_TMA = 32, SK_TMA128 = 33, SK_TMA64 = 34,     // B built from the node tensors in shared memory
  SK_TMAF = 40, SK_TMAF128 = 41, SK_TMAF64 = 42,  // B pieces formed in HBM, loaded by TMA
  SK_TMAC = 48, SK_TMAC128 = 49, SK_TMAC64 = 50,  // B formed in HBM as complex64, split on chip
  SK_TMAP = 56, SK_TMAP128 = 57, SK_TMAP64 = 58,  // the same, one persistent CTA per SM
  SK_TMAPA = 64, SK_TMAPA128 = 65, SK_TMAPA64 = 66,  // persistent, A read as complex64 and split on chip too
  SK_TMAPF = 72, SK_TMAPF128 = 73, SK_TMAPF64 = 74,  // persistent, A and B pieces by TMA (B formed in HBM,
                                                     // once per slice for a ket tensor)
  SK_TMAPFA = 80, SK_TMAPFA128 = 81, SK_TMAPFA64 = 82  // persistent, A complex64 split on chip, B pieces by TMA
};
inline bool sk_is_tma(int k) { return k >= SK_TMA && k <= SK_TMAPFA64 && (k & 7) <= 2; }
inline bool sk_tma_persist(int k) { return sk_is_tma(k) && k >= SK_TMAP; }
// the kernel reads its input as complex64 and splits it on chip
inline bool sk_tma_c64a(int k) { return sk_is_tma(k) && ((k >= SK_TMAPA && k < SK_TMAPF) || k >= SK_TMAPFA); }
// the kernel reads its input as the bf16 pieces its producer writes (else as complex64)
inline bool sk_reads_pieces(int k) { return sk_is_tma(k) && !sk_tma_c64a(k); }
inline int sk_tma_bmode(int k) { return k >= SK_TMAPF ? 0 : k >= SK_TMAC ? 2 : k >= SK_TMAF ? 0 : 1; }
inline int sk_tma_bn(int k) { return (k & 7) == 1 ? 128 : (k & 7) == 2 ? 64 : 0; }
std::vector<int> step_kernels(const tn_plan *p, tn_precision prec);
bool step_kernel_ok(const StepParams &s, tn_precision prec, int k);

tn_path_opts tn_default_opts();
int64_t plan_ws_bytes(const tn_plan *p, int kind, int64_t chunk, int64_t slices);
tn_status ws_ensure(tn_plan *p, Workspace &w, int kind, cudaStream_t st);
tn_status ws_ensure_sized(tn_plan *p, Workspace &w, int kind, int64_t chunk, int64_t slices, cudaStream_t st);
// buffer sizes of a workspace, and a workspace laid out (256-byte aligned, not owned) in given memory
enum { WS_BITS, WS_BRA64, WS_BRA32, WS_KET64, WS_KET32, WS_GWORK, WS_T0, WS_T1, WS_CBUF, WS_RES, WS_ERR, WS_NBUF };
struct WsSizes {
  int64_t b[WS_NBUF];
  int64_t total;                                  // with 256-byte alignment of every buffer
};
WsSizes ws_sizes(const tn_plan *p, int kind, int64_t chunk, int64_t slices);
void ws_carve(Workspace &w, void *base, const WsSizes &z, int64_t chunk, int64_t slices, cudaStream_t st);
bool is_device_ptr(const void *p);
// the operands of step j: the plan's ket and bra buffers, or for a double-layer step the absorbed
// tensor's buffer and the unit operand (kind 0: complex128, 1: complex64) with its arguments
void step_operands(const tn_plan *p, size_t j, int kind, const void *ket, const void *bra, const ContractArgs &a,
                   const void *&kj, const void *&bj, ContractArgs &aj);
// one contraction step j with kernel k (with the overlap formation that kernel needs); no host sync
cudaError_t enqueue_step(const tn_plan *p, const Workspace &w, size_t j, int k, tn_precision prec,
                         const ContractArgs &a, const void *ket, const void *bra, const void *tin, void *tout,
                         const OutDesc &od, cudaStream_t st);
tn_status check_err_words(const int *err);   // the two error words of a workspace, read on the host
tn_status enqueue_chunk(tn_plan *p, Workspace &w, const uint64_t *bits_dev, int64_t nb, tn_precision prec,
                        const std::vector<int> &ks, double2 *res_dev, cudaStream_t st, int64_t slice_begin = 0,
                        int64_t slice_end = -1);
void ws_release(DevMem &mem, Workspace &w);
// amplitudes, or with a slice range the FP64 partial sums over slices [slice_begin, slice_end)
tn_status run_amplitudes(tn_plan *p, Workspace &w, const uint64_t *bits, int64_t n, tn_precision prec,
                         tn_c128 *out, cudaStream_t st, int64_t slice_begin = 0, int64_t slice_end = -1);
tn_status run_half(const Half &h, int n_qubits, double2 *base, int items, const int64_t *node_off_dev,
                   const uint64_t *bits_dev, int words, double2 *gwork, int *errflag, cudaStream_t st,
                   int *rank_out_dev, const double2 *init_vec_dev, int64_t item_stride = 0);

// tracing: events around launches, attributed to a kernel kind
// the contraction step whose launches the ProfScopes of this thread belong to, while it lives
struct ProfStep {
  explicit ProfStep(int step);
  ~ProfStep();
};
struct ProfScope {
  int slot = -1;
  cudaStream_t st = 0;
  ProfScope(const char *kind, cudaStream_t stream, double bytes, double flops);
  ~ProfScope();
};

/*
 * tn.h -- C ABI of the GB300 tensor-network-states amplitude library.
 *
 * The library computes amplitudes a(s) = <s| U |0...0> of a quantum circuit U
 * on an arbitrary connected qubit graph with the tensor-network-states method
 * of Guo, Zhao and Huang (arXiv:2011.02621):
 *
 *   tn_build             graph + gate list (problem statement; Eq. gatesplit)
 *   tn_evolve_two_sided  two-sided evolution with SVD compression
 *                        (Eqs. result1, result2, svd, svd2; Fig. 2a)
 *   tn_path              cuts + contraction path by Algorithm 1 (supplement)
 *   tn_amplitudes        batched bra evolution, overlap network (Eq. overlap),
 *                        sliced path-ordered contraction, sum over slices
 *
 * plus a serving loop (tn_server_*) that batches amplitude requests for
 * resident plans.
 *
 * Conventions shared by every call:
 *  - Every call returns a tn_status; nothing is thrown across the ABI.
 *    tn_last_error() gives a thread-local message for the last failure.
 *  - Inputs are copied during the call; the caller keeps ownership of every
 *    pointer it passes. Handles are owned by the library and released with
 *    the matching tn_*_free.
 *  - Device memory is obtained through the caller's tn_allocator when one is
 *    given (e.g. PyTorch's caching allocator), else with cudaMalloc / cudaFree.
 *  - Streams are the caller's (a cudaStream_t passed as void*; NULL = the
 *    legacy default stream). Work on one tn_plan must be serialised by the
 *    caller (one stream, or host synchronisation between calls): the plan
 *    owns a single workspace.
 *  - Asynchronous CUDA errors surface as TN_ERR_CUDA at the next call that
 *    synchronises. A bounded device-side wait that expires gives
 *    TN_ERR_TIMEOUT.
 *  - The library needs a CUDA device of compute capability 10.3 (sm_103a)
 *    for every call that touches the device; there is no CPU fallback.
 *    tn_path_search and tn_gate_split are host-only.
 */
#ifndef TN_H
#define TN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TN_OK = 0,
  TN_ERR_ARG = 1,        /* bad argument (NULL, negative size, out of range) */
  TN_ERR_GRAPH = 2,      /* graph disconnected, gate on a non-edge, qubit out of range */
  TN_ERR_OOM = 3,        /* allocator returned NULL or admission refused */
  TN_ERR_NO_PATH = 4,    /* Algorithm 1 found no path within its limits */
  TN_ERR_STATE = 5,      /* call order (e.g. tn_path before tn_evolve_two_sided) */
  TN_ERR_CUDA = 6,       /* a CUDA runtime error */
  TN_ERR_TIMEOUT = 7,    /* a bounded wait expired */
  TN_ERR_UNSUPPORTED = 8 /* shape outside the implemented limits */
} tn_status;

typedef struct { double re, im; } tn_c128;

/* Qubit graph G = {V, E} (paper: lattice geometry paragraph). Qubits are
 * 0..n_qubits-1; edges[2*i], edges[2*i+1] are the endpoints of edge i (its id
 * is i). The graph must be connected and simple. */
typedef struct {
  int32_t n_qubits;
  int32_t n_edges;
  const int32_t *edges;
} tn_graph;

/* One gate. arity 1: m[0..3] is the 2x2 matrix (row-major, rows = outputs).
 * arity 2: m[0..15] is the 4x4 matrix in the basis |q[0] q[1]>, q[0] the
 * high bit; {q[0], q[1]} must be an edge. cycle >= 1 orders the gates into
 * cycles for the two-sided split; gates are applied in array order. */
typedef struct {
  int32_t cycle;
  int32_t arity;
  int32_t q[2];
  tn_c128 m[16];
} tn_gate;

/* Device allocator. alloc returns device memory of `bytes` usable on
 * `stream` (NULL on failure); free releases it (stream-ordered). */
typedef struct {
  void *(*alloc)(size_t bytes, void *stream, void *ctx);
  void (*free)(void *ptr, size_t bytes, void *stream, void *ctx);
  void *ctx;
} tn_allocator;

/* Arithmetic of the contraction GEMMs (the evolution SVDs, the truncation
 * decision and the cross-slice sum are always FP64). */
typedef enum {
  TN_FP64 = 0,   /* complex128 tensors, FP64 SIMT GEMMs */
  TN_FP32 = 1,   /* complex64 tensors, FP32 SIMT GEMMs */
  TN_TF32 = 2,   /* complex64 tensors, single-pass TF32 tcgen05 GEMMs, FP32 accumulate */
  TN_TF32X3 = 3, /* complex64, compensated hi/lo TF32 (3 products), FP32 accumulate */
  TN_BF16X3 = 4, /* complex64, compensated hi/lo BF16 (3 products), FP32 accumulate */
  TN_BF16X6 = 5, /* complex64, three-piece BF16 split (6 products, ~24-bit products), FP32 accumulate */
  TN_TF32X6 = 6  /* complex64, three-piece TF32 split (6 products), FP32 accumulate */
} tn_precision;

typedef struct tn_circuit tn_circuit;
typedef struct tn_plan tn_plan;

/* Options of tn_path (supplement: Assumptions 1-3, Algorithm 1; cutting). */
typedef struct {
  int32_t max_rank;      /* M of Assumption 2 (max open legs of an intermediate);
                            0 = smallest M >= max degree that completes within max_states */
  int32_t boundary_only; /* 1 = Assumption 1 (start at nodes of degree < max degree); 0 = any node */
  int32_t connected;     /* 1 = Assumption 3 (almost-connected partial paths); 0 = unconstrained */
  int64_t max_states;    /* cap on Algorithm 1 expansions; 0 = 4,000,000 */
  int32_t n_cuts;        /* -1 = automatic (fit max_intermediate); >= 0 = this many cuts */
  const int32_t *cut_edges; /* explicit cut list (edge ids); overrides n_cuts when n_cut_edges > 0 */
  int32_t n_cut_edges;
  int64_t max_intermediate; /* automatic cuts keep every intermediate <= this many elements
                               per (bitstring, slice); 0 = 2^24 */
  double mem_budget_bytes;  /* workspace budget of tn_amplitudes; 0 = 8 GiB */
  int32_t no_merge;         /* 1 = one network node per qubit; 0 = merge boundary nodes of degree
                               <= 2 into a neighbour first (exact; see tn_path) */
  int32_t layers;           /* 0 or 1 = the overlap network of Eq. overlap (one node per qubit);
                               2 = the double-layer network (see tn_path) */
  double byte_weight;       /* 0 = Algorithm 1's score (complex MACs); w > 0 adds w x (input +
                               output elements) per step, for steps bound by memory traffic
                               (w ~ compute rate / bandwidth in complex MACs per element) */
} tn_path_opts;

/* Summary of a plan. All counts are per amplitude unless stated. */
typedef struct {
  int32_t n_qubits;
  int32_t n_steps;            /* pairwise contraction steps (n_nodes - 1) */
  int32_t n_cuts;
  int64_t n_slices;           /* product of the cut edges' dimensions */
  double score;               /* Algorithm 1 score of the path (complex MACs per slice) */
  double cmacs;               /* complex multiply-adds over all steps and slices */
  double flops;               /* 8 * cmacs (real flops) */
  double bytes_c64;           /* algorithmic bytes: sum over steps of 8*(M*K + M*N), times slices */
  int64_t max_intermediate;   /* largest intermediate, elements per (bitstring, slice) */
  int64_t states_expanded;    /* Algorithm 1 pops */
  int32_t max_rank_used;      /* M that Algorithm 1 ran with */
  int32_t chunk_bitstrings;   /* bitstrings per device batch */
  int64_t workspace_bytes;    /* device workspace for the widest precision */
  int32_t n_nodes;            /* nodes of the contracted network (n_qubits minus merged nodes) */
} tn_plan_info;

/* Build a circuit: validates the graph (connected, simple, endpoints in
 * range) and the gates (2-qubit gates only on edges), and copies both.
 * Host only; no device memory is touched. `alloc` may be NULL.
 * Errors: TN_ERR_ARG, TN_ERR_GRAPH. */
tn_status tn_build(const tn_graph *g, const tn_gate *gates, int64_t n_gates,
                   const tn_allocator *alloc, tn_circuit **out);

/* Two-sided evolution (Fig. 2a): gates of cycles 1..split_cycle act on
 * |0...0> (the ket half, evolved now on the device in FP64 by
 * Eqs. result1/result2 + svd/svd2); gates of cycles split_cycle+1.. are
 * recorded as the bra program (their transposes, last to first) that
 * tn_amplitudes runs per bitstring. Single-qubit gates are fused into the
 * next two-qubit gate on that qubit in each half's processing order.
 * Compression keeps singular values > cutoff_rel * s_0, at most chi_max
 * (0 = no cap); bond shapes are the static structural bounds
 * min(chi, dim*chi_o, 2*prod(other legs)) with rank deficits zero-padded.
 * May be called again with other arguments (plans made before are invalid).
 * Errors: TN_ERR_ARG, TN_ERR_CUDA, TN_ERR_OOM, TN_ERR_UNSUPPORTED. */
tn_status tn_evolve_two_sided(tn_circuit *c, int32_t split_cycle, int32_t chi_max,
                              double cutoff_rel, void *cuda_stream);

/* Bond compression of both halves (the SVD step after every two-qubit gate).
 *   TN_COMPRESS_ONE_SIDED (default): Eqs. svd/svd2 as the paper states them. The endpoint
 *     with fewer rows 2*prod(other legs) (ties: q[0]) is decomposed, A^sv <- U, and S V^H is
 *     absorbed into the other endpoint; the kept singular values are those of A^sv alone.
 *   TN_COMPRESS_TWO_SIDED: a variant the paper does not use. The kept singular values are
 *     those of the local product A^sv A^other^T, which is what a thin QR of both endpoints
 *     followed by an SVD of R_sv R_other^T yields. A truncated bond is then the best
 *     approximation of that rank of the pair (Eckart-Young), and its rank is that of the
 *     product. The device runs it as two entries of the same gate kernel per two-qubit gate.
 *     The first applies the gate and decomposes the other endpoint exactly (cutoff 0, no chi
 *     cap), so that endpoint becomes an isometry. The second is an identity gate that
 *     decomposes A^sv with the keep rule. Same endpoint rule and the same structural bond
 *     shapes as the one-sided form. Untruncated, both give the same amplitudes.
 * Host only. Takes effect at the next tn_evolve_two_sided, which rebuilds the programs when
 * the mode changed (plans made before are then invalid). Errors: TN_ERR_ARG. */
typedef enum { TN_COMPRESS_ONE_SIDED = 0, TN_COMPRESS_TWO_SIDED = 1 } tn_compress;
tn_status tn_set_compression(tn_circuit *c, int32_t mode);

/* Cap on the sweeps of the one-sided Jacobi SVD (Eqs. svd/svd2) of every compression of both
 * halves: 1..1000, 0 = the default (60). A compression that has not converged within the cap sets
 * the error word of its launch, and the call that ran it returns TN_ERR_TIMEOUT (the bounded
 * loop ends; the context stays usable). Host only; takes effect at once for the bra half of later
 * amplitude calls and for the next tn_evolve_two_sided. Errors: TN_ERR_ARG. */
tn_status tn_set_svd_sweeps(tn_circuit *c, int32_t max_sweeps);

/* Host-only inspection of the gate program of one half (side 0 = ket, 1 = bra) that
 * tn_evolve_two_sided(c, split_cycle, chi_max, cutoff_rel) builds with the circuit's
 * compression mode, from the structural bond bounds (no rank probe, no device work), for CPU
 * models of the evolution kernels. Call once with NULL entries/mats to get *n_entries, then
 * with entries[n_entries * TN_PROG_ENTRY_LEN] and mats[n_entries * TN_PROG_MAT_LEN]. Entry i,
 * in processing order, is
 *   a two-qubit entry (op 2): op, k, l, edge, sv_is_k, din, chi_o, n = din*chi_o, dout, m_k,
 *     m_l, pk, pl (positions of the edge among k's and l's legs), off_k, off_l, id; mats: P and
 *     Q as 16 complex each (re, im; P[(s'*2 + s)*4 + a], s' the output and s the input value of
 *     the physical index, a the term of Eq. gatesplit), then the cutoff. On the node tensors
 *     [sigma, legs in increasing edge id] it forms X_k = P A^k and X_l = Q A^l, the shared leg
 *     becoming (a_old, a) at index a_old*chi_o + a (Eqs. result1/result2). It takes the SVD of
 *     the endpoint named by sv_is_k, matricised as (sigma, other legs) x (bond). It keeps
 *     keep = min(#{s_j > cutoff * s_0}, dout) singular values, largest first, and zero-pads to
 *     dout. Then A^sv <- U and A^other <- X_other (S V^H)^T (Eqs. svd/svd2).
 *   a single-qubit entry (op 1, the tail of single-qubit gates with no later two-qubit gate):
 *     op, q, -1, ..., off at [13]; mats: the 2x2 matrix as 4 complex, applied to sigma.
 * The ket starts from |0...0>, the bra from the bitstring's basis state.
 * Errors: TN_ERR_ARG. */
#define TN_PROG_ENTRY_LEN 16
#define TN_PROG_MAT_LEN 66
tn_status tn_program_inspect(const tn_circuit *c, int32_t split_cycle, int32_t chi_max, double cutoff_rel,
                             int32_t side, int64_t *entries, double *mats, int64_t *n_entries);

/* Structural bond dimensions after evolution: side 0 = ket, 1 = bra;
 * out[n_edges]. Errors: TN_ERR_STATE before tn_evolve_two_sided. */
tn_status tn_circuit_bond_dims(const tn_circuit *c, int32_t side, int32_t *out);

/* Cuts and contraction path (supplement, Algorithm 1 with Assumptions 1-3;
 * cutting as in the overlap paragraph), compiled into static per-step
 * shapes and uploaded. `opts` may be NULL (defaults). `info` may be NULL.
 * Unless opts->no_merge, boundary nodes are first merged into a neighbour: a
 * node v of degree <= 2 whose other legs are no wider than its edge a to u is
 * contracted with u over a, separately and exactly (FP64) on the ket and on
 * every bitstring's bra, giving one node with a physical index of 4 (or 8)
 * values; the overlap network and the amplitudes are unchanged, the path
 * search and the contraction see fewer, no larger nodes.
 * With opts->layers == 2 the network is the double-layer one: node q is qubit q's ket tensor,
 * node n_qubits + q its bra tensor, the two joined by an edge of dimension 2 (the physical
 * index), ket bonds between ket nodes and bra bonds between bra nodes; network edge ids are
 * e (ket bond of circuit edge e), n_edges + e (its bra bond) and 2 n_edges + q (qubit q's
 * physical index). The sums are those of Eq. overlap without forming the per-qubit overlap
 * tensors first, so the amplitudes are the same; each step absorbs one ket tensor (the same for
 * every bitstring) or one bra tensor. Unless opts->no_merge, partial paths are then joined
 * (supplement, the discussion of Assumption 3): where the path absorbs two tensors of the same
 * layer in a row that share one edge not cut, the pair is contracted with each other first
 * (ket pairs once per batch in FP64; bra pairs per bitstring, in FP64 for TN_FP64 and in FP32
 * for the complex64 precisions, whose contraction carries FP32-level products) and absorbed in one step,
 * when that lowers both the complex multiply-adds and the elements the steps read and write; the
 * amplitudes are the same sums grouped otherwise and no intermediate grows. Explicit cut_edges
 * are not accepted (TN_ERR_UNSUPPORTED); automatic cuts are. The path search holds at most 256 nodes, so the
 * double-layer network takes every circuit tn_build accepts (at most 128 qubits).
 * Errors: TN_ERR_STATE, TN_ERR_NO_PATH, TN_ERR_ARG, TN_ERR_CUDA, TN_ERR_OOM, TN_ERR_UNSUPPORTED. */
tn_status tn_path(tn_circuit *c, const tn_path_opts *opts, tn_plan **out, tn_plan_info *info);

/* Host-only estimate of the plan tn_path(opts) would make after
 * tn_evolve_two_sided(c, split_cycle, chi_max, cutoff_rel): the same gate programs with their
 * structural bond bounds (no device work and no rank probe, so a bond can be wider than an
 * evolved circuit's), the same network, path, cuts and compiled steps, every table checked
 * against the node tensors and the item strides as tn_path does. Fills `info`; c is not
 * modified and needs no evolution. Errors: TN_ERR_ARG, TN_ERR_NO_PATH, TN_ERR_UNSUPPORTED. */
tn_status tn_plan_estimate(const tn_circuit *c, int32_t split_cycle, int32_t chi_max, double cutoff_rel,
                           const tn_path_opts *opts, tn_plan_info *info);

/* Host-only inspection of the compiled steps of the plan tn_plan_estimate describes (same
 * arguments), for CPU models of the contraction and checks of the plan compiler. Call once with
 * NULL layout/steps/tables to get *n_steps and *n_tables, then with buffers of these sizes:
 *   layout[8 + 2*n_qubits + 2*n_edges]: max intermediate (item stride), slices, steps, ket and
 *     bra item elements of the network (with merged nodes), 1 if nodes were merged, ket and bra
 *     item elements of the halves; per qubit its ket and bra node offsets; per edge its ket and
 *     bra bond. A node tensor is [sigma, legs in increasing edge id], complex, row-major.
 *   steps[n_steps * TN_STEP_DESC_LEN]: per step M, K, N, layer (0 overlap node, 1 ket tensor,
 *     2 bra tensor of a double-layer plan), n_rest, ket_off, ket_sig, bra_off, bra_sig, phys,
 *     the table offsets of ocol, bka, bkb, bna, bnb, sa, sb, then TN_PLAN_MAXREST rest dims
 *     (slowest first) and TN_PLAN_MAXREST rest output strides.
 *   tables[n_tables]: the int32 tables.
 * A step computes, per item (bitstring b, slice l): with x = ket + ket_off + sa[l] and
 * y = bra_b + bra_off + sb[l], C[k][n] = sum_{s < phys} x[bka[k] + bna[n] + s*ket_sig] *
 * y[bkb[k] + bnb[n] + s*bra_sig]; out[orow(m) + ocol[n]] = sum_k in[m*K + k] C[k][n], orow(m)
 * the mixed-radix digits of m over the rest dims times their strides. Step 0 writes C[0][n] at
 * ocol[n]. For layer 1 (2) steps y (x) is the unit operand [1, 0]. The amplitude is the sum over
 * slices of the last step's out[0].
 * Errors: TN_ERR_ARG, TN_ERR_NO_PATH, TN_ERR_UNSUPPORTED. */
#define TN_PLAN_MAXREST 32
#define TN_STEP_DESC_LEN (17 + 2 * TN_PLAN_MAXREST)
tn_status tn_plan_inspect(const tn_circuit *c, int32_t split_cycle, int32_t chi_max, double cutoff_rel,
                          const tn_path_opts *opts, int64_t *layout, int64_t *steps, int32_t *tables,
                          int64_t *n_steps, int64_t *n_tables);

/* Plan details: order[max(n_qubits, n_nodes)] (contraction order of the network's nodes,
 * each named by its representative qubit, then -1 for the merged qubits; for a double-layer
 * plan its n_nodes node ids, q for qubit q's ket tensor and n_qubits + q for its bra tensor, a
 * joined node named by its first tensor), cuts[n_cuts] (circuit edge ids; network edge ids for a
 * double-layer plan), steps[3*n_steps] = (M, K, N) per step per slice.
 * Any pointer may be NULL. */
tn_status tn_plan_details(const tn_plan *p, int32_t *order, int32_t *cuts, int64_t *steps);

/* Amplitudes of n bitstrings. bits: n rows of ceil(n_qubits/64) uint64 words,
 * bit q of word q/64 = s_q; host or device memory. out: n tn_c128, host or
 * device memory. Runs the bra program per bitstring (FP64), the overlap
 * network and the sliced contraction in `prec`, and the FP64 slice sum, in
 * device batches of info.chunk_bitstrings on `cuda_stream`; returns after
 * the results are in `out` (the stream is synchronised).
 * Errors: TN_ERR_ARG, TN_ERR_CUDA, TN_ERR_OOM, TN_ERR_UNSUPPORTED. */
tn_status tn_amplitudes(tn_plan *p, const uint64_t *bits, int64_t n, tn_precision prec,
                        tn_c128 *out, void *cuda_stream);

/* Partial amplitudes: for each bitstring the FP64 sum over the slices [slice_begin, slice_end)
 * of the plan's cut network only (0 <= slice_begin <= slice_end <= info.n_slices; an empty range
 * gives zeros). Summing the results over a partition of [0, n_slices) gives tn_amplitudes up to
 * the order of the FP64 additions. This is how slices are sharded over ranks when a job has fewer
 * bitstrings than ranks (cutting, overlap paragraph: the amplitude is the sum over the cut
 * indices). Same arguments, memory rules and errors as tn_amplitudes. */
tn_status tn_amplitudes_slices(tn_plan *p, const uint64_t *bits, int64_t n, tn_precision prec,
                               int64_t slice_begin, int64_t slice_end, tn_c128 *out, void *cuda_stream);

/* tn_amplitudes without device allocation. The paper has no counterpart: this is for callers
 * that must not allocate device memory while they run -- a process whose own pool already holds
 * the GPU's memory and accounts for every byte, a real-time or embedded host limited to a budget
 * fixed at start-up, or code running inside an allocator callback, which must not re-enter the
 * allocator. Same arguments, results and precisions as tn_amplitudes; every scratch buffer is
 * carved from one static device array of 32 MiB that each GPU loading the library holds until
 * the process exits. No cudaMalloc, cudaFree or allocator callback is called.
 *  - The first call on a device looks up the array's device address (a CUDA runtime query,
 *    once per device, with that device current); make that first call before any stream
 *    capture begins.
 *  - Call it with the plan's device current (the device its circuit was evolved on): the array
 *    used is the current device's, so another current device is refused with TN_ERR_ARG.
 *  - Batches are sized to fit the array; a plan whose single bitstring and single slice need
 *    more than 32 MiB is rejected with TN_ERR_UNSUPPORTED (use tn_amplitudes, or plan with a
 *    smaller max_intermediate).
 *  - All calls share the array and it keeps the previous call's contents; each call clears the
 *    words it needs at zero and writes every other buffer before reading it. Calls whose work
 *    overlaps on the GPU (other streams, other threads) race on the array: serialise them. */
tn_status tn_amplitudes_static(tn_plan *p, const uint64_t *bits, int64_t n, tn_precision prec,
                               tn_c128 *out, void *cuda_stream);

/* ---- kernel autotuning and batched circuits ------------------------------- */

/* Step kernels (values written by tn_autotune / tn_plan_kernels, one per contraction step):
 * 0 shape heuristic (SIMT), 1-3 SIMT tiles 64x64 / 128x16 / 256x4 (rows x columns),
 * 4 SIMT streaming (K, N <= 16), 5 SIMT streaming with K and N fixed at compile time,
 * 6 SIMT one-CTA-per-item reduction (small outputs), 7 SIMT few-rows kernel (M <= 16, M*K <= 2048,
 * one thread per output column), 8 SIMT box-tiled streaming step (K*N <= 4096, N <= 256, the plan's
 * row tiles), 16 tcgen05 with the operand split in the kernel (TF32, TF32x3, BF16x3, TF32x6), and
 * the TMA-fed tcgen05 kernels (BF16x6), each with the tile picked by shape / 128-column /
 * 64-column tiles: 32 / 33 / 34 building the overlap operand in shared memory from the node
 * tensors, 40 / 41 / 42 loading it as bf16 pieces formed in HBM, 48 / 49 / 50 reading it as
 * complex64 formed in HBM and splitting it on chip; the persistent forms (one CTA per SM walking
 * the output tiles, K < 256): 56 / 57 / 58 as 48-50, 64 / 65 / 66 the same with the step's input
 * read as complex64 and split on chip (the previous step then writes complex64, not bf16 pieces),
 * 72 / 73 / 74 with the operand as bf16 pieces formed in HBM (once per slice for a ket tensor),
 * 80 / 81 / 82 the same with the input read as complex64. The paper has no counterpart: which
 * kernel runs a pairwise contraction is an implementation choice that changes no result beyond
 * rounding. */
enum { TN_KERNEL_SIMT = 0, TN_KERNEL_SIMT_BOX = 8, TN_KERNEL_TC = 16, TN_KERNEL_TMA = 32, TN_KERNEL_TMA128 = 33,
       TN_KERNEL_TMA64 = 34, TN_KERNEL_TMA_LOADB = 40, TN_KERNEL_TMA_LOADB128 = 41, TN_KERNEL_TMA_LOADB64 = 42,
       TN_KERNEL_TMA_C64B = 48, TN_KERNEL_TMA_C64B128 = 49, TN_KERNEL_TMA_C64B64 = 50,
       TN_KERNEL_PERSIST = 56, TN_KERNEL_PERSIST128 = 57, TN_KERNEL_PERSIST64 = 58,
       TN_KERNEL_PERSIST_C64 = 64, TN_KERNEL_PERSIST_C64_128 = 65, TN_KERNEL_PERSIST_C64_64 = 66,
       TN_KERNEL_PERSIST_LOADB = 72, TN_KERNEL_PERSIST_LOADB128 = 73, TN_KERNEL_PERSIST_LOADB64 = 74,
       TN_KERNEL_PERSIST_C64_LOADB = 80, TN_KERNEL_PERSIST_C64_LOADB128 = 81, TN_KERNEL_PERSIST_C64_LOADB64 = 82 };

/* Time every kernel that supports each contraction step of the plan in precision `prec`, on the
 * plan's workspace with a batch of min(n_bits, chunk) bitstrings (n_bits = 0: the full chunk),
 * and keep the fastest per step (the shape heuristic's kernel unless another is >= 3% faster).
 * A kernel that reads its input as bf16 pieces is charged the previous step's time writing them;
 * a second pass re-picks each step in its final output format.
 * The choice is stored in the plan for `prec` and used by every later amplitude, server and batch
 * call on it. kernels (may be NULL): info.n_steps entries, the chosen kernel per step.
 * Synchronises the stream. Errors: TN_ERR_ARG, TN_ERR_STATE, TN_ERR_CUDA, TN_ERR_OOM, TN_ERR_TIMEOUT. */
tn_status tn_autotune(tn_plan *p, tn_precision prec, int64_t n_bits, void *cuda_stream, int32_t *kernels);

/* The kernels the plan runs in `prec` (tuned, else the shape heuristic), info.n_steps entries. */
tn_status tn_plan_kernels(const tn_plan *p, tn_precision prec, int32_t *kernels);

/* Set the plan's kernels for `prec`: info.n_steps TN_KERNEL_* values, each supporting its step
 * (TN_ERR_ARG otherwise, and nothing changes); NULL returns to the shape heuristic. */
tn_status tn_plan_set_kernels(tn_plan *p, tn_precision prec, const int32_t *kernels);

typedef struct tn_batch tn_batch;

/* Several circuits (their plans, each with its own batch of bitstrings; shapes may differ) as one
 * CUDA graph. bits: every circuit's bitstrings concatenated in plan order, circuit i taking
 * n_bits[i] rows of ceil(n_qubits_i/64) words; host or device memory, copied. Each circuit runs
 * its bitstrings in chunks of its plan's batch size (info.chunk_bitstrings). The circuits are
 * grouped, in order, into waves whose workspaces fit hbm_budget_bytes side by side (0: one wave
 * of all); the waves run one after another and share one workspace arena, so the batch holds the
 * largest wave's workspaces plus the bitstrings and results (allocated through the first
 * circuit's allocator). It runs every circuit once on `cuda_stream` to validate it and captures
 * the whole batch (per wave one independent branch per circuit: bra evolution, overlap,
 * contraction with the plan's kernels, FP64 slice sum) into one graph; a graph of more than
 * 100000 kernels is refused (TN_ERR_UNSUPPORTED). Plans and circuits must outlive the batch;
 * re-evolving a circuit invalidates it. The paper has no counterpart: this is the batching of
 * many circuits into one launch.
 * Errors: TN_ERR_ARG, TN_ERR_STATE, TN_ERR_CUDA, TN_ERR_OOM, TN_ERR_TIMEOUT, TN_ERR_UNSUPPORTED. */
tn_status tn_batch_create(tn_plan *const *plans, int32_t n_plans, const uint64_t *bits, const int64_t *n_bits,
                          tn_precision prec, double hbm_budget_bytes, void *cuda_stream, tn_batch **out);

/* Replace every circuit's bitstrings (same layout and counts as at creation); stream-ordered. */
tn_status tn_batch_set_bits(tn_batch *b, const uint64_t *bits, void *cuda_stream);

/* One launch of the batch's graph on `cuda_stream`; asynchronous. Errors: TN_ERR_STATE, TN_ERR_CUDA. */
tn_status tn_batch_run(tn_batch *b, void *cuda_stream);

/* All amplitudes of the last run, concatenated in plan order, into out (host or device); reads
 * the circuits' error words and synchronises the stream. Errors: TN_ERR_CUDA, TN_ERR_TIMEOUT. */
tn_status tn_batch_read(tn_batch *b, tn_c128 *out, void *cuda_stream);

/* Kernel nodes in the graph and device bytes the batch holds. Either pointer may be NULL. */
tn_status tn_batch_info(const tn_batch *b, int64_t *graph_kernels, int64_t *device_bytes);

void tn_batch_free(tn_batch *b);

/* Kernel launches issued since the last reset (all threads). */
int64_t tn_launch_count(int32_t reset);

/* Per-kernel timing (tracing): while enabled, every launch is bracketed by
 * CUDA events on its own stream and attributed to a kernel kind together
 * with its algorithmic bytes and flops. tn_profile_enable(1) clears the
 * records; tn_profile_read synchronises the recorded events and returns kind
 * `idx` (TN_ERR_ARG past the last kind): name (NUL-terminated, at most
 * name_len bytes), launches, total milliseconds, algorithmic bytes and flops.
 * on = 2 keeps one record per kind and contraction step: the launches of
 * the step at index i of the lists of tn_plan_details and tn_plan_kernels
 * are named "<kind>#i". on = 0 stops recording. */
tn_status tn_profile_enable(int32_t on);
tn_status tn_profile_read(int32_t idx, char *name, int32_t name_len, int64_t *launches, double *ms,
                          double *bytes, double *flops);

void tn_circuit_free(tn_circuit *c);
void tn_plan_free(tn_plan *p);
const char *tn_last_error(void);

/* ---- host-only pieces, usable without a GPU ------------------------------ */

/* Eq. gatesplit: O[(k',l'),(k,l)] = sum_s P[k',k,s] Q[l',l,s] with chi_o = the
 * number of singular values > 1e-12 s_0 of O regrouped as (k',k) x (l',l).
 * m: 16 entries (4x4 row-major). P, Q: 16 entries each, index (a*2+b)*4+s for
 * P[a][b][s]; unused s are zero. */
tn_status tn_gate_split(const tn_c128 *m, tn_c128 *P, tn_c128 *Q, int32_t *chi_o);

/* Algorithm 1 on an arbitrary graph with per-edge dimensions `dims`
 * (n_edges entries, >= 1). order[n_qubits] receives the path, *score its
 * score (Cost = product of the dims of all legs of both tensors). Graphs of
 * up to 256 nodes (tn_cut_search likewise; circuits hold at most 128 qubits).
 * Errors: TN_ERR_ARG, TN_ERR_GRAPH, TN_ERR_NO_PATH, TN_ERR_UNSUPPORTED. */
tn_status tn_path_search(const tn_graph *g, const double *dims, const tn_path_opts *opts,
                         int32_t *order, double *score, int64_t *states_expanded);

/* Cuts and path of tn_path on an arbitrary graph with per-edge dimensions:
 * order[n_qubits], cuts[<= n_edges] (edge ids, *n_cuts of them) and the total
 * complex multiply-adds (slices x score of the cut network). Host only.
 * Errors: TN_ERR_ARG, TN_ERR_GRAPH, TN_ERR_NO_PATH. */
tn_status tn_cut_search(const tn_graph *g, const double *dims, const tn_path_opts *opts, int32_t *order,
                        int32_t *cuts, int32_t *n_cuts, double *total_cmacs);

/* The network tn_path contracts, on an arbitrary graph with per-edge ket and bra dimensions:
 * boundary nodes merged into neighbours (unless opts->no_merge; explicit cut edges are never
 * merged away), then Algorithm 1 and the cuts as in tn_path. owner[n_qubits]: the node each qubit
 * belongs to, named by its representative qubit; *n_nodes nodes; order[*n_nodes]: the contraction
 * order (representative qubits); *n_cuts and *total_cmacs (slices x score) may be NULL. Host only.
 * Errors: TN_ERR_ARG, TN_ERR_GRAPH, TN_ERR_NO_PATH. */
tn_status tn_merge_search(const tn_graph *g, const int32_t *ket_dims, const int32_t *bra_dims,
                          const tn_path_opts *opts, int32_t *owner, int32_t *n_nodes, int32_t *order, int32_t *n_cuts,
                          double *total_cmacs);

/* ---- serving loop (continuous batching over resident plans) -------------- */

typedef struct tn_server tn_server;

typedef struct {
  double hbm_budget_bytes;  /* admission budget for in-flight work; 0 = 16 GiB */
  int32_t max_inflight;     /* concurrently running requests; 0 = 4 */
  int32_t n_streams;        /* device streams the worker threads use; 0 = max_inflight */
} tn_server_cfg;

typedef struct {
  int64_t submitted, completed, failed, rejected;
  int64_t amplitudes;
  double busy_seconds;       /* wall time with >= 1 request in flight */
  double p50_latency_s, p99_latency_s;   /* completion - submission, over completed requests */
  double max_inflight_seen;
  double peak_admitted_bytes;
  int64_t cancelled;         /* requests removed from the queue by tn_server_cancel */
} tn_server_stats;

/* Create a server; its worker threads (min(max_inflight, n_streams) of them), each with its
 * own stream and workspaces, take the oldest request whose device memory fits the budget next
 * to the batches in flight, merge into it the queued requests of the same plan and precision
 * (continuous batching, up to the plan's batch size), and run them as one device batch of the
 * tn_amplitudes path. Free the server before the plans it served. Errors: TN_ERR_ARG, TN_ERR_CUDA. */
tn_status tn_server_create(const tn_server_cfg *cfg, tn_server **out);

/* Queue a request (the bits are copied; out must stay valid until the ticket
 * completes). The plan must stay alive until then and may be shared by
 * several requests (each running request gets its own workspace).
 * Errors: TN_ERR_ARG, TN_ERR_OOM (footprint above the whole budget). */
tn_status tn_server_submit(tn_server *s, tn_plan *p, const uint64_t *bits, int64_t n,
                           tn_precision prec, tn_c128 *out, uint64_t *ticket);

/* Wait for a ticket; timeout_ms < 0 waits forever. Returns the request's
 * own status, or TN_ERR_TIMEOUT if it has not completed in time. */
tn_status tn_server_wait(tn_server *s, uint64_t ticket, int64_t timeout_ms);

/* Cancel a request that is still queued (no worker has taken it): it is removed, its output is
 * not written and its ticket is forgotten (a later tn_server_wait on it gives TN_ERR_ARG). The
 * paper has no counterpart: this is the serving loop's request management. A request that is
 * running or complete cannot be cancelled: TN_ERR_STATE (wait for it). Errors: TN_ERR_ARG
 * (unknown ticket), TN_ERR_STATE. */
tn_status tn_server_cancel(tn_server *s, uint64_t ticket);

tn_status tn_server_stats_get(tn_server *s, tn_server_stats *st);

/* Drains queued work, joins the workers and frees the server. */
void tn_server_free(tn_server *s);

#ifdef __cplusplus
}
#endif
#endif /* TN_H */

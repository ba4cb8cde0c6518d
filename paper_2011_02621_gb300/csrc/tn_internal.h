// Internal declarations shared by the host code (host.cpp, server.cpp) and the
// CUDA translation units (evolve.cu, contract.cu, tc_gemm.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tn.h"

#define TN_MAXLEG 8     // legs (incident edges) per node
#define TN_MAXREST 32   // rest legs of one contraction step

// ---------------------------------------------------------------------------
// evolution (Eqs. result1/result2, svd/svd2)
// ---------------------------------------------------------------------------
// Node tensors of one half live in a per-item region; node q at offset
// node_off[q] (complex elements), layout [sigma, leg_0, ..., leg_{n-1}]
// row-major with legs in increasing edge id.
struct GateParams {
  int64_t off_k, off_l;        // node offsets within an item region
  int nk, nl;                  // leg counts of k and l
  int dk[TN_MAXLEG];           // dims of k's legs before the gate (leg pk has din)
  int dl[TN_MAXLEG];
  int pk, pl;                  // position of the shared edge among the legs
  int din, chi_o, dout;        // bond dim before the gate, gate rank, bond bound after
  int sv_is_k;                 // 1: SVD node k and absorb S V into l; 0: the reverse
  int m_k, m_l, n;             // rows of the matricised k and l (2*prod other legs), n = din*chi_o
  int use_smem;                // work buffers in dynamic shared memory
  double cutoff;               // keep singular values > cutoff * s_0
  double2 P[16];               // P[s'][s][a] at (s'*2+s)*4+a  (Eq. gatesplit)
  double2 Q[16];
  int64_t work_stride;         // per-item global work size (complex elements) when !use_smem
  int id;                      // position in the half's gate program (reported when the SVD fails)
  int max_sweeps;              // cap on Jacobi sweeps (0: the default, 60); then the error word is set
};

struct Apply1Params {
  int64_t off;                 // node offset
  int64_t size_rest;           // prod of the node's leg dims
  double2 u[4];                // 2x2, rows = outputs
};

// work (complex elements) the gate kernel needs per item
int64_t gate_work_elems(const GateParams &g);

cudaError_t launch_init_product(double2 *base, int64_t item_stride, int items, const int64_t *node_off_dev,
                                int n_qubits, const uint64_t *bits, int words, const double2 *init_vec,
                                cudaStream_t st);
// rank_out (nullable): item 0 writes the numerical rank of its SVD there
cudaError_t launch_gate(const GateParams &g, double2 *base, int64_t item_stride, int items,
                        double2 *gwork, int *errflag, int *rank_out, cudaStream_t st);
cudaError_t launch_apply1(const Apply1Params &a, double2 *base, int64_t item_stride, int items, cudaStream_t st);
cudaError_t launch_to_c64(const double2 *src, float2 *dst, int64_t n, cudaStream_t st);

// Merging node v into its neighbour u through their shared edge a, on one half (ket or bra), in
// FP64 and exactly: out[p_u, p_v, legs_u \ a, legs_v \ a] = sum_a U[p_u, legs_u] V[p_v, legs_v].
// Element offsets are within one item's region; the rest legs are listed in output order.
#define TN_MAXMLEGS 8          // rest legs of a merged pair in the overlap network's merging policy
#define TN_MERGE_MAXLEGS 16    // rest legs per operand a merge can describe (joined double-layer nodes)
struct MergeParams {
  int64_t u_off, v_off, out_off, out_size;
  int64_t su_p, sv_p;                   // physical-index strides in U and V
  int64_t su_a, sv_a;                   // strides of the shared leg a in U and V
  int pu, pv, da;                       // physical values of U and V, dim of a on this half
  int nu, nv;                           // rest legs of U and V
  int du[TN_MERGE_MAXLEGS], dv[TN_MERGE_MAXLEGS];       // their dims
  int64_t su[TN_MERGE_MAXLEGS], sv[TN_MERGE_MAXLEGS];   // their strides in U and V
};
cudaError_t launch_merge(const MergeParams &m, double2 *base, int64_t item_stride, int64_t items, cudaStream_t st);
cudaError_t launch_merge(const MergeParams &m, float2 *base, int64_t item_stride, int64_t items, cudaStream_t st);
cudaError_t launch_pack_bits(const uint64_t *src, uint64_t *dst, int64_t n_words, cudaStream_t st);

// ---------------------------------------------------------------------------
// contraction (Eq. overlap; path-ordered steps of Algorithm 1; cutting)
// ---------------------------------------------------------------------------
// One absorption step (TTGT with both transposes folded into the kernels):
//   T_out[item][orow(m) + ocol[n]] = sum_k T_in[item][m*K + k] * C[k][n],
//   C[k][n] = sum_sigma ket[ka(k,n) + sigma*ket_sig] * bra_b[kb(k,n) + sigma*bra_sig]   (Eq. overlap)
// item = bitstring * n_slices + slice. Every intermediate is stored in the layout its consumer
// reads as a row-major [M][K] matrix (rest legs, then shared legs): the producer of step j
// writes element (m, n) at orow(m) + ocol[n], where orow decomposes m over the rest legs of
// step j (mixed radix, last fastest) with their strides in step j+1's layout.
struct StepParams {
  int64_t M, K, N;
  int n_rest;
  int rest_pow2;                // 1: every rest dim is a power of two (decompose with shifts)
  int rest_dim[TN_MAXREST];     // rest legs of step j, slowest first
  int rest_log2[TN_MAXREST];    // log2 of the dims when rest_pow2
  int rest_ostride[TN_MAXREST]; // their strides in the output layout
  int64_t ket_off, ket_sig;     // node tensor offset / physical-index stride in the ket buffer
  int64_t bra_off, bra_sig;     // same in one bitstring's bra region
  int64_t phys;                 // values of the node's physical index (2; 4 or 8 for merged nodes)
  // offsets of the int32 tables in the plan's table buffer
  int64_t t_ocol, t_bka, t_bkb, t_bna, t_bnb, t_sa, t_sb;
  // Row tiles of the box-tiled streaming kernel (SIMT_BOX; 0 = the step has none): box_tm rows
  // m = t * box_tm + r, r < box_tm, whose input rows are one contiguous block and whose output
  // offsets split as orow(t * box_tm) + orow(r) (box_tm is aligned to the rest digits).
  // t_wperm: box_tm * N entries (r << 16 | n), the tile's outputs in increasing output offset.
  int box_tm;
  int64_t t_wperm;
};

struct ContractArgs {
  const int32_t *tab;           // plan table buffer (device)
  int64_t n_slices;             // slices per bitstring in this launch group
  int64_t slice0;               // first slice of the group (global slice index)
  int64_t items;                // bitstrings_in_chunk * n_slices
  int64_t t_stride;             // elements per item in T buffers
  int64_t bra_stride;           // elements per bitstring region of the bra buffer
};

// Where a producer writes an intermediate: fmt 0 = complex64 (or complex128 on the FP64
// path) at [item * t_stride + offset]; fmt 1 = three bf16 planes (pieces of every real, see
// the tensor-core step), plane q at (uint32 *)p + q * plane_u32, the (re, im) pair of a complex
// element as one uint32 at [item * t_stride + offset].
struct OutDesc {
  void *p;
  int fmt;
  int64_t plane_u32;
};

// bf16 pieces operand for a TMA load: plane q at (uint16 *)base + q * plane_elems, item i at
// + i * item_elems (bf16 elements)
struct Pieces {
  const void *base;
  int64_t plane_elems, item_elems;
};

// precision-templated launchers (R = double or float)
template <typename R>
cudaError_t launch_form(const StepParams &s, const ContractArgs &a, const void *ket, const void *bra,
                        const OutDesc &out, cudaStream_t st);
template <typename R>
cudaError_t launch_step(const StepParams &s, const ContractArgs &a, const void *ket, const void *bra,
                        const void *t_in, const OutDesc &out, cudaStream_t st, int variant = 0);
// SIMT step kernels: the shape heuristic or one kernel forced (the autotuner's candidates)
enum SimtVariant { SIMT_AUTO = 0, SIMT_T64 = 1, SIMT_T128 = 2, SIMT_T256 = 3, SIMT_STREAM = 4, SIMT_FIXED = 5,
                   SIMT_SMALL = 6, SIMT_NARROW = 7, SIMT_BOX = 8 };
bool simt_variant_ok(const StepParams &s, int variant, bool fp64);
// the box-tiled streaming step (stream.cu): thin steps with K * N <= TN_BOX_MAXKN, N <= TN_BOX_MAXN
#define TN_BOX_MAXKN 4096
#define TN_BOX_MAXN 256
#define TN_BOX_ROWS_ELEMS 6144   // box_tm * (2 K + N) at most (two input tiles and one output tile)
template <typename R>
cudaError_t launch_step_box(const StepParams &s, const ContractArgs &a, const void *ket, const void *bra,
                            const void *t_in, const OutDesc &out, cudaStream_t st);
// out[b] (+)= sum over the group's slices, in slice order, in FP64 (accumulate: add to out)
template <typename R>
cudaError_t launch_slice_sum(const void *res, int64_t items_stride, int64_t n_bits, int64_t n_slices,
                             int accumulate, double2 *out, cudaStream_t st);

// the overlap tensor of one step for every item, complex64, [N][K] per item (K contiguous)
cudaError_t launch_form_c(const StepParams &s, const ContractArgs &a, const float2 *ket, const float2 *bra,
                          float2 *cbuf, int64_t c_stride, cudaStream_t st);
// tensor-core step (tcgen05): prec = TN_TF32 .. TN_TF32X6; B from launch_form_c's buffer
cudaError_t launch_step_tc(int prec, const StepParams &s, const ContractArgs &a, const float2 *cbuf,
                           int64_t c_stride, const float2 *t_in, float2 *t_out, int *errflag, cudaStream_t st);
bool tc_step_supported(const StepParams &s);
// the overlap tensor of one step in its real embedding, split into three bf16 planes
cudaError_t launch_form_b_pieces(const StepParams &s, const ContractArgs &a, const float2 *ket, const float2 *bra,
                                 const Pieces &B, cudaStream_t st);
// TMA-fed tcgen05 step (BF16x6) from pre-split A and B pieces
// bn: output tile width in real columns (128 or 64; 0 picks by shape). The B operand: with cbuf
// (the overlap tensor as complex64 [N][K], c_stride elements apart, from launch_form_c; item i
// reads copy i % c_items, c_items 0 meaning one copy per item) the kernel splits it in shared
// memory; else with ket and bra (the complex64 node tensors) it builds it in shared memory; else
// it loads B, formed by launch_form_b_pieces.
cudaError_t launch_step_tma(const StepParams &s, const ContractArgs &a, const Pieces &A, const Pieces &B,
                            const OutDesc &out, int *err, cudaStream_t st, int bn = 0, const float2 *ket = nullptr,
                            const float2 *bra = nullptr, const float2 *cbuf = nullptr, int64_t c_stride = 0,
                            int64_t c_items = 0);
bool tma_step_supported(const StepParams &s);
// Long contractions on the TMA-fed BF16x6 step take 64-column tiles: the tensor core adds its
// products into an FP32 accumulator with truncation, so the error grows with the number of MMAs
// summed into one accumulator; a 64-column tile spreads the order-0 products over 7 TMEM
// accumulators instead of 3 (measured relative to rms |a| against FP64: the 4x5 grid at 14 cycles,
// K up to 4096, 8.7e-6 -> 4.9e-6; the 53-qubit overlap network, K = 256, up to 1.05e-5 on 128-column
// tiles, above the 1e-5 the amplitudes must meet).
#define TN_TMA_LONG_K 256

// launch accounting
void tn_count_launch(int64_t k);

// Two-sided circuit evolution on the device, batched over items (bitstrings):
// product-state initialisation (Eq. initialstate), fused two-qubit gate
// application + one-sided Jacobi SVD compression + absorption (Eqs. result1,
// result2, svd, svd2), and single-qubit applications. FP64 throughout.
#include <cuda_runtime.h>
#include <math.h>

#include "tn_internal.h"
#include "tn_smem.h"

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // a*b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// Row-major view of a node tensor [sigma, legs...] with one distinguished leg `pos`.
struct NodeView {
  int nleg, pos;
  int dims[TN_MAXLEG];
  int64_t stride[TN_MAXLEG];
  int64_t sig;   // stride of sigma = prod of leg dims
};

__device__ void make_view(NodeView &v, const int *dims, int nleg, int pos, int pos_dim) {
  v.nleg = nleg;
  v.pos = pos;
  int64_t s = 1;
  for (int j = nleg - 1; j >= 0; --j) {
    v.dims[j] = (j == pos) ? pos_dim : dims[j];
    v.stride[j] = s;
    s *= v.dims[j];
  }
  v.sig = s;
}

// offset of the "other legs" multi-index o (legs != pos, last fastest)
__device__ __forceinline__ int64_t other_offset(const NodeView &v, int64_t o) {
  int64_t off = 0;
  for (int j = v.nleg - 1; j >= 0; --j) {
    if (j == v.pos) continue;
    int d = v.dims[j];
    off += (o % d) * v.stride[j];
    o /= d;
  }
  return off;
}

struct WorkLayout {
  int R, C;          // Jacobi operand Y is R x C, column-major
  int64_t y, xo, w, vp, sig, rank, total;
};

__host__ __device__ inline WorkLayout work_layout(const GateParams &g) {
  WorkLayout L;
  int m_sv = g.sv_is_k ? g.m_k : g.m_l;
  int m_o = g.sv_is_k ? g.m_l : g.m_k;
  if (g.n <= m_sv) { L.R = m_sv; L.C = g.n; } else { L.R = g.n; L.C = m_sv; }
  L.y = 0;
  L.xo = L.y + (int64_t)L.R * L.C;
  L.w = L.xo + (int64_t)m_o * g.n;
  L.vp = L.w + (int64_t)L.C * L.C;
  L.sig = L.vp + (int64_t)g.dout * g.n;
  L.rank = L.sig + L.C;
  L.total = L.rank + L.C;
  return L;
}

__host__ __device__ inline int C_of(const WorkLayout &L) { return L.C; }

constexpr int GATE_THREADS = 128;
constexpr int MAX_SWEEPS = 60;

// TPI threads per item (128: one item per CTA; 32, 16, 8 or 4: 32 / TPI items per warp, 128 / TPI
// per CTA, for small matrices): X_k = P A^k, X_l = Q A^l (Eqs. result1/result2), SVD of the
// smaller-row endpoint by parallel one-sided (Hestenes) Jacobi, keep s_j > cutoff*s_0 (at
// most dout, zero-padded to dout), A^sv <- U, A^other <- X_other (S V)^T (Eqs. svd/svd2).
// With several items in a warp every lane runs the same instruction stream: the rotation
// parameters of the pairs of all those items come from one pass of the FP64 square roots and
// divisions that dominate the work of small matrices.
template <int TPI>
__device__ __forceinline__ void item_sync() {
  if (TPI <= 32) __syncwarp(); else __syncthreads();
}

// sum of x over the TPI lanes of this item's aligned lane group (TPI <= 32)
template <int TPI>
__device__ __forceinline__ double group_sum(double x) {
#pragma unroll
  for (int o = TPI / 2; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

template <int TPI>
__global__ void __launch_bounds__(GATE_THREADS) gate_kernel(GateParams g, double2 *base, int64_t item_stride,
                                                            double2 *gwork, int *errflag, int items, int *rank_out) {
  extern __shared__ double2 smem[];
  constexpr bool SUB = TPI <= 32;                 // items within one warp (no block-wide barrier)
  constexpr int GPB = GATE_THREADS / TPI;         // items per block
  const int grp = threadIdx.x / TPI;
  const int item = blockIdx.x * GPB + grp;
  const int tid = threadIdx.x % TPI;
  const int lane = tid & 31, warp = tid >> 5, nwarp = TPI >= 32 ? TPI / 32 : 1;
  // a warp whose first item is past the end has nothing to do; a group past the end inside a
  // live warp runs along (its lanes take part in the warp's shuffles) on the last item's data
  // and writes nothing
  if (SUB && blockIdx.x * GPB + (int)(threadIdx.x / 32) * (32 / (SUB ? TPI : 32)) >= items) return;
  const bool valid = item < items;
  double2 *A = base + (int64_t)(valid ? item : items - 1) * item_stride;
  const WorkLayout L = work_layout(g);
  double2 *work = g.use_smem ? smem + (int64_t)grp * L.total : gwork + (int64_t)item * g.work_stride;
  double2 *Y = work + L.y, *Xo = work + L.xo, *W = work + L.w, *Vp = work + L.vp;
  double *sig = reinterpret_cast<double *>(work + L.sig);
  int *rank = reinterpret_cast<int *>(work + L.rank);
  int *colof = rank + C_of(L);   // inverse of rank (the rank slots hold 4 ints per column)

  NodeView vk, vl;
  make_view(vk, g.dk, g.nk, g.pk, g.din);
  make_view(vl, g.dl, g.nl, g.pl, g.din);
  const int n = g.n, chi_o = g.chi_o;
  const bool ytrans = !(n <= (g.sv_is_k ? g.m_k : g.m_l));   // Y = X^H

  // ---- gate application into the work buffers
  for (int side = 0; side < 2; ++side) {
    const bool is_k = (side == 0);
    const NodeView &v = is_k ? vk : vl;
    const double2 *Pm = is_k ? g.P : g.Q;
    const double2 *An = A + (is_k ? g.off_k : g.off_l);
    const int m = is_k ? g.m_k : g.m_l;
    const bool is_sv = (is_k == (g.sv_is_k != 0));
    const int64_t O = m / 2;
    const int64_t total = (int64_t)m * n;
    for (int64_t idx = tid; idx < total; idx += TPI) {
      int r = (int)(idx / n), c = (int)(idx % n);
      int sp = (int)(r / O);
      int64_t o = r % O;
      int a = c / chi_o, s = c % chi_o;
      int64_t off = other_offset(v, o) + (int64_t)a * v.stride[v.pos];
      double2 x = cmul(Pm[(sp * 2 + 0) * 4 + s], An[off]);
      x = cfma(Pm[(sp * 2 + 1) * 4 + s], An[off + v.sig], x);
      if (is_sv) {
        if (!ytrans) Y[(int64_t)c * m + r] = x;              // Y = X, column-major
        else Y[(int64_t)r * n + c] = cconj(x);               // Y = X^H, column-major
      } else {
        Xo[(int64_t)r * n + c] = x;
      }
    }
  }
  const int R = L.R, C = L.C;
  for (int64_t idx = tid; idx < (int64_t)C * C; idx += TPI) {
    int i = (int)(idx % C), j = (int)(idx / C);
    W[idx] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  item_sync<TPI>();

  // ---- parallel one-sided Jacobi (round-robin pairing)
  // rotation threshold: |<y_p, y_q>| > tol * |y_p| |y_q| with tol = 2 sqrt(R) eps (the rounding
  // level of the column dot products). Pairs whose smaller column is at the rounding level of the
  // whole matrix (|y|^2 <= 16 R eps^2 ||Y||_F^2: a singular value below the untruncated cutoff)
  // are left alone, and a sweep counts as unconverged only for a rotation above 8 tol, so the
  // iteration ends on rounding-dominated pairs (exactly degenerate spectra are common here).
  __shared__ int s_rot_a[GPB];
  __shared__ double s_fro_a[GPB];
  __shared__ double s_part_a[GPB][TPI >= 32 ? TPI / 32 : 1];
  int &s_rot = s_rot_a[grp];
  double &s_fro = s_fro_a[grp];
  double *s_part = s_part_a[grp];
  {
    double f = 0;
    for (int64_t idx = tid; idx < (int64_t)L.R * L.C; idx += TPI) f = fma(Y[idx].x, Y[idx].x, fma(Y[idx].y, Y[idx].y, f));
    if constexpr (SUB) {
      f = group_sum<TPI>(f);
      if (tid == 0) s_fro = f;
    } else {
      for (int o = 16; o; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
      if (lane == 0) s_part[warp] = f;
      item_sync<TPI>();
      if (tid == 0) {
        double t = 0;
        for (int w = 0; w < TPI / 32; ++w) t += s_part[w];
        s_fro = t;
      }
    }
    item_sync<TPI>();
  }
  const double eps = 2.220446049250313e-16;
  const double tol = 2.0 * sqrt((double)L.R) * eps;
  const double floor_ab = 1e-30 * s_fro;
  const double floor_col = 16.0 * (double)L.R * eps * eps * s_fro;
  const int Cp = (C + 1) & ~1;
  const int rounds = Cp - 1;
  bool converged = (C <= 1);
  const int sweep_cap = g.max_sweeps > 0 ? g.max_sweeps : MAX_SWEEPS;
  // the loop runs while any item of the warp (SUB) or the item (TPI 128) is unconverged: a
  // converged item's pairs are below the rotation threshold and stay as they are
  for (int sweep = 0; sweep < sweep_cap; ++sweep) {
    if (SUB ? __all_sync(0xffffffffu, converged) : converged) break;
    if (tid == 0) s_rot = 0;
    item_sync<TPI>();
    for (int rd = 0; rd < rounds; ++rd) {
      if constexpr (SUB) {
        // items of TPI lanes inside a warp: the round's column pairs (disjoint columns) side by
        // side, LP lanes per pair, each lane summing rows r = sub, sub + LP, ... and the pair's
        // lanes reducing with shuffles inside their aligned LP-lane segment
        const int npairs = Cp / 2;
        int LP = TPI;
        while (LP > 1 && LP * npairs > TPI) LP >>= 1;
        const int sub = tid & (LP - 1), slot = tid / LP;
        for (int pi0 = 0; pi0 < npairs; pi0 += TPI / LP) {
          const int pi = pi0 + slot;
          int p = 0, q = 0;
          if (pi == 0) { p = rd; q = Cp - 1; }
          else { p = (rd + pi) % (Cp - 1); q = (rd - pi + (Cp - 1)) % (Cp - 1); }
          const bool act = pi < npairs && p < C && q < C;
          double2 *yp = Y + (int64_t)p * R, *yq = Y + (int64_t)q * R;
          double al = 0, be = 0, gr = 0, gi = 0;
          if (act) {
            for (int r = sub; r < R; r += LP) {
              double2 a = yp[r], b = yq[r];
              al = fma(a.x, a.x, fma(a.y, a.y, al));
              be = fma(b.x, b.x, fma(b.y, b.y, be));
              gr = fma(a.x, b.x, fma(a.y, b.y, gr));    // conj(a) * b
              gi = fma(a.x, b.y, fma(-a.y, b.x, gi));
            }
          }
          for (int o = LP >> 1; o; o >>= 1) {
            al += __shfl_xor_sync(0xffffffffu, al, o);
            be += __shfl_xor_sync(0xffffffffu, be, o);
            gr += __shfl_xor_sync(0xffffffffu, gr, o);
            gi += __shfl_xor_sync(0xffffffffu, gi, o);
          }
          if (!act) continue;
          const double ga = sqrt(gr * gr + gi * gi);
          const double nab = sqrt(al * be);
          if (!(ga > tol * nab) || nab <= floor_ab || ga == 0.0 || fmin(al, be) <= floor_col) continue;
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
          const double2 e = make_double2(gr / ga, -gi / ga);       // conj(gamma)/|gamma|
          for (int r = sub; r < R; r += LP) {
            double2 a = yp[r], b = cmul(yq[r], e);
            yp[r] = make_double2(cs * a.x - sn * b.x, cs * a.y - sn * b.y);
            yq[r] = make_double2(sn * a.x + cs * b.x, sn * a.y + cs * b.y);
          }
          double2 *wp = W + (int64_t)p * C, *wq = W + (int64_t)q * C;
          for (int r = sub; r < C; r += LP) {
            double2 a = wp[r], b = cmul(wq[r], e);
            wp[r] = make_double2(cs * a.x - sn * b.x, cs * a.y - sn * b.y);
            wq[r] = make_double2(sn * a.x + cs * b.x, sn * a.y + cs * b.y);
          }
          if (sub == 0 && ga > 8.0 * tol * nab) s_rot = 1;
        }
      } else {
      for (int pi = warp; pi < Cp / 2; pi += nwarp) {
        int p, q;
        if (pi == 0) { p = rd; q = Cp - 1; }
        else { p = (rd + pi) % (Cp - 1); q = (rd - pi + (Cp - 1)) % (Cp - 1); }
        if (p >= C || q >= C) continue;
        double2 *yp = Y + (int64_t)p * R, *yq = Y + (int64_t)q * R;
        double al = 0, be = 0, gr = 0, gi = 0;
        for (int r = lane; r < R; r += 32) {
          double2 a = yp[r], b = yq[r];
          al = fma(a.x, a.x, fma(a.y, a.y, al));
          be = fma(b.x, b.x, fma(b.y, b.y, be));
          gr = fma(a.x, b.x, fma(a.y, b.y, gr));    // conj(a) * b
          gi = fma(a.x, b.y, fma(-a.y, b.x, gi));
        }
        for (int o = 16; o; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          gr += __shfl_xor_sync(0xffffffffu, gr, o);
          gi += __shfl_xor_sync(0xffffffffu, gi, o);
        }
        double ga = sqrt(gr * gr + gi * gi);
        const double nab = sqrt(al * be);
        if (!(ga > tol * nab) || nab <= floor_ab || ga == 0.0 || fmin(al, be) <= floor_col) continue;
        double zeta = (be - al) / (2.0 * ga);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        double2 e = make_double2(gr / ga, -gi / ga);       // conj(gamma)/|gamma|
        for (int r = lane; r < R; r += 32) {
          double2 a = yp[r], b = cmul(yq[r], e);
          yp[r] = make_double2(cs * a.x - sn * b.x, cs * a.y - sn * b.y);
          yq[r] = make_double2(sn * a.x + cs * b.x, sn * a.y + cs * b.y);
        }
        double2 *wp = W + (int64_t)p * C, *wq = W + (int64_t)q * C;
        for (int r = lane; r < C; r += 32) {
          double2 a = wp[r], b = cmul(wq[r], e);
          wp[r] = make_double2(cs * a.x - sn * b.x, cs * a.y - sn * b.y);
          wq[r] = make_double2(sn * a.x + cs * b.x, sn * a.y + cs * b.y);
        }
        if (lane == 0 && ga > 8.0 * tol * nab) s_rot = 1;
      }
      }
      item_sync<TPI>();
    }
    converged = (s_rot == 0);
    item_sync<TPI>();
  }
  if (!converged && tid == 0 && valid) atomicCAS(errflag, 0, 1 + g.id);   // first failing gate, 1-based

  // ---- singular values, descending ranks, truncation count
  if constexpr (SUB) {
    for (int j = 0; j < C; ++j) {
      const double2 *yj = Y + (int64_t)j * R;
      double s2 = 0;
      for (int r = tid; r < R; r += TPI) s2 = fma(yj[r].x, yj[r].x, fma(yj[r].y, yj[r].y, s2));
      s2 = group_sum<TPI>(s2);
      if (tid == 0) sig[j] = sqrt(s2);
    }
  } else {
    for (int j = warp; j < C; j += nwarp) {
      const double2 *yj = Y + (int64_t)j * R;
      double s2 = 0;
      for (int r = lane; r < R; r += 32) s2 = fma(yj[r].x, yj[r].x, fma(yj[r].y, yj[r].y, s2));
      for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) sig[j] = sqrt(s2);
    }
  }
  item_sync<TPI>();
  __shared__ double s_max_a[GPB];
  __shared__ int s_keep_a[GPB];
  double &s_max = s_max_a[grp];
  int &s_keep = s_keep_a[grp];
  if (tid == 0) {
    double mx = 0;
    for (int j = 0; j < C; ++j) mx = fmax(mx, sig[j]);
    int kc = 0;
    for (int j = 0; j < C; ++j) kc += (sig[j] > g.cutoff * mx) ? 1 : 0;
    s_max = mx;
    s_keep = kc < g.dout ? kc : g.dout;
    if (rank_out && item == 0 && valid) {
      // numerical rank: singular values above the rounding level of the column norms
      const double thr = 4.0 * sqrt((double)R) * 2.220446049250313e-16 * mx;
      int nr = 0;
      for (int j = 0; j < C; ++j) nr += (sig[j] > thr) ? 1 : 0;
      *rank_out = nr;
    }
  }
  for (int j = tid; j < C; j += TPI) {
    int rk = 0;
    for (int i = 0; i < C; ++i) rk += (sig[i] > sig[j] || (sig[i] == sig[j] && i < j)) ? 1 : 0;
    rank[j] = rk;
    colof[rk] = j;
  }
  item_sync<TPI>();
  const int keep = s_keep;
  const int dout = g.dout;

  // ---- V' = S V^H rows (dout x n), zero beyond keep
  for (int64_t idx = tid; idx < (int64_t)dout * n; idx += TPI) Vp[idx] = make_double2(0, 0);
  item_sync<TPI>();
  for (int j = 0; j < C; ++j) {
    int t = rank[j];
    if (t >= keep) continue;
    for (int c = tid; c < n; c += TPI) {
      double2 v;
      if (!ytrans) { double2 w = W[(int64_t)j * C + c]; v = make_double2(sig[j] * w.x, -sig[j] * w.y); }
      else { v = cconj(Y[(int64_t)j * R + c]); }
      Vp[(int64_t)t * n + c] = v;
    }
  }

  // ---- A^sv <- U (new layout, leg pos has dout)
  {
    const bool svk = g.sv_is_k != 0;
    NodeView nv;
    make_view(nv, svk ? g.dk : g.dl, svk ? g.nk : g.nl, svk ? g.pk : g.pl, dout);
    double2 *An = A + (svk ? g.off_k : g.off_l);
    const int m = svk ? g.m_k : g.m_l;
    const int64_t O = m / 2;
    const int64_t total = (int64_t)m * dout;
    for (int64_t idx = tid; idx < total; idx += TPI) {
      int r = (int)(idx / dout), t = (int)(idx % dout);
      double2 u = make_double2(0, 0);
      if (t < keep) {
        const int j = colof[t];
        if (!ytrans) {
          double2 y = Y[(int64_t)j * R + r];
          double inv = sig[j] > 0 ? 1.0 / sig[j] : 0.0;
          u = make_double2(y.x * inv, y.y * inv);
        } else {
          u = W[(int64_t)j * C + r];
        }
      }
      int sp = (int)(r / O);
      int64_t o = r % O;
      if (valid) An[sp * nv.sig + other_offset(nv, o) + (int64_t)t * nv.stride[nv.pos]] = u;
    }
  }
  item_sync<TPI>();

  // ---- A^other <- X_other V'^T
  {
    const bool svk = g.sv_is_k != 0;
    NodeView nv;
    make_view(nv, svk ? g.dl : g.dk, svk ? g.nl : g.nk, svk ? g.pl : g.pk, dout);
    double2 *An = A + (svk ? g.off_l : g.off_k);
    const int m = svk ? g.m_l : g.m_k;
    const int64_t O = m / 2;
    const int64_t total = (int64_t)m * dout;
    for (int64_t idx = tid; idx < total; idx += TPI) {
      int r = (int)(idx / dout), t = (int)(idx % dout);
      double2 acc = make_double2(0, 0);
      const double2 *xr = Xo + (int64_t)r * n, *vt = Vp + (int64_t)t * n;
      for (int c = 0; c < n; ++c) acc = cfma(xr[c], vt[c], acc);
      int sp = (int)(r / O);
      int64_t o = r % O;
      if (valid) An[sp * nv.sig + other_offset(nv, o) + (int64_t)t * nv.stride[nv.pos]] = acc;
    }
  }
}

// product state: basis states from `bits` (|0> without bits), or the given per-qubit 2-vectors
__global__ void init_product_kernel(double2 *base, int64_t item_stride, int items, const int64_t *node_off,
                                    int nq, const uint64_t *bits, int words, const double2 *init_vec) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)items * nq) return;
  int item = (int)(idx / nq), q = (int)(idx % nq);
  double2 *A = base + (int64_t)item * item_stride + node_off[q];
  if (init_vec) {
    A[0] = init_vec[2 * q];
    A[1] = init_vec[2 * q + 1];
    return;
  }
  int b = 0;
  if (bits) b = (int)((bits[(int64_t)item * words + (q >> 6)] >> (q & 63)) & 1ull);
  A[0] = make_double2(b == 0 ? 1.0 : 0.0, 0.0);
  A[1] = make_double2(b == 1 ? 1.0 : 0.0, 0.0);
}

__global__ void apply1_kernel(Apply1Params a, double2 *base, int64_t item_stride, int items) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)items * a.size_rest) return;
  int64_t item = idx / a.size_rest, r = idx % a.size_rest;
  double2 *A = base + item * item_stride + a.off;
  double2 x0 = A[r], x1 = A[r + a.size_rest];
  A[r] = cfma(a.u[0], x0, cmul(a.u[1], x1));
  A[r + a.size_rest] = cfma(a.u[2], x0, cmul(a.u[3], x1));
}

__global__ void to_c64_kernel(const double2 *src, float2 *dst, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

__global__ void copy_words_kernel(const uint64_t *src, uint64_t *dst, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

}  // namespace

int64_t gate_work_elems(const GateParams &g) { return work_layout(g).total; }

namespace {

template <int TPI>
cudaError_t launch_items_per_warp(const GateParams &g, const WorkLayout &L, double2 *base, int64_t item_stride,
                                  int items, double2 *gwork, int *errflag, int *rank_out, cudaStream_t st) {
  constexpr int GPB = GATE_THREADS / TPI;
  const size_t smem = (size_t)GPB * L.total * sizeof(double2);
  if (smem > 48 * 1024) {
    const int lim = tn_smem_optin<gate_kernel<TPI>>();
    if (lim < 0 || (size_t)lim < smem) return cudaErrorInvalidValue;
  }
  gate_kernel<TPI><<<(items + GPB - 1) / GPB, GATE_THREADS, smem, st>>>(g, base, item_stride, gwork, errflag, items,
                                                                        rank_out);
  tn_count_launch(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gate(const GateParams &g, double2 *base, int64_t item_stride, int items, double2 *gwork,
                        int *errflag, int *rank_out, cudaStream_t st) {
  if (items <= 0) return cudaSuccess;
  const WorkLayout L = work_layout(g);
  // small matrices: items inside one warp, as many lanes each as a Jacobi round's pairs cover
  // over all rows (at least 4, at most 32), 128 / lanes items per CTA in shared memory
  const bool warp_per_item = g.use_smem && L.C <= 16 && L.R <= 256 && 4 * L.total * sizeof(double2) <= 96 * 1024;
  if (warp_per_item) {
    const int npairs = ((L.C + 1) & ~1) / 2;
    int tpi = 4;
    while (tpi < 32 && tpi < npairs * L.R) tpi <<= 1;
    while (tpi < 32 && (size_t)(GATE_THREADS / tpi) * L.total * sizeof(double2) > 96 * 1024) tpi <<= 1;
    switch (tpi) {
      case 4: return launch_items_per_warp<4>(g, L, base, item_stride, items, gwork, errflag, rank_out, st);
      case 8: return launch_items_per_warp<8>(g, L, base, item_stride, items, gwork, errflag, rank_out, st);
      case 16: return launch_items_per_warp<16>(g, L, base, item_stride, items, gwork, errflag, rank_out, st);
      default: return launch_items_per_warp<32>(g, L, base, item_stride, items, gwork, errflag, rank_out, st);
    }
  }
  const size_t smem = g.use_smem ? (size_t)L.total * sizeof(double2) : 0;
  if (smem > 48 * 1024) {
    const int lim = tn_smem_optin<gate_kernel<128>>();
    if (lim < 0 || (size_t)lim < smem) return cudaErrorInvalidValue;
  }
  gate_kernel<128><<<items, GATE_THREADS, smem, st>>>(g, base, item_stride, gwork, errflag, items, rank_out);
  tn_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_init_product(double2 *base, int64_t item_stride, int items, const int64_t *node_off_dev,
                                int n_qubits, const uint64_t *bits, int words, const double2 *init_vec,
                                cudaStream_t st) {
  int64_t total = (int64_t)items * n_qubits;
  if (total <= 0) return cudaSuccess;
  init_product_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(base, item_stride, items, node_off_dev,
                                                                       n_qubits, bits, words, init_vec);
  tn_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_apply1(const Apply1Params &a, double2 *base, int64_t item_stride, int items, cudaStream_t st) {
  int64_t total = (int64_t)items * a.size_rest;
  if (total <= 0) return cudaSuccess;
  apply1_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(a, base, item_stride, items);
  tn_count_launch(1);
  return cudaGetLastError();
}

// Merged node tensors: one output element o of one item per thread, o fastest, so that when the
// merged tensor is small (tens of elements for a joined pair of bra tensors) a block covers
// several items; the sum over the shared leg in index order, in the precision of V2 (FP64, or
// FP32 for the complex64 forms' per-bitstring bra pairs).
template <typename V2>
__global__ void merge_kernel(MergeParams m, V2 *base, int64_t item_stride, int64_t items) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= items * m.out_size) return;
  const int64_t item = idx / m.out_size, o = idx % m.out_size;
  int64_t r = o, iu = 0, iv = 0;
  for (int j = m.nv - 1; j >= 0; --j) {
    iv += (r % m.dv[j]) * m.sv[j];
    r /= m.dv[j];
  }
  for (int j = m.nu - 1; j >= 0; --j) {
    iu += (r % m.du[j]) * m.su[j];
    r /= m.du[j];
  }
  iv += (r % m.pv) * m.sv_p;
  iu += (r / m.pv) * m.su_p;
  const V2 *U = base + item * item_stride + m.u_off + iu;
  const V2 *V = base + item * item_stride + m.v_off + iv;
  V2 acc;
  acc.x = 0;
  acc.y = 0;
  for (int x = 0; x < m.da; ++x) {
    const V2 u = U[x * m.su_a], v = V[x * m.sv_a];
    acc.x = fma(u.x, v.x, fma(-u.y, v.y, acc.x));
    acc.y = fma(u.x, v.y, fma(u.y, v.x, acc.y));
  }
  base[item * item_stride + m.out_off + o] = acc;
}

template <typename V2>
cudaError_t launch_merge_t(const MergeParams &m, V2 *base, int64_t item_stride, int64_t items, cudaStream_t st) {
  if (items <= 0 || m.out_size <= 0) return cudaSuccess;
  const int64_t blocks = (items * m.out_size + 255) / 256;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  merge_kernel<V2><<<(unsigned)blocks, 256, 0, st>>>(m, base, item_stride, items);
  tn_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_merge(const MergeParams &m, double2 *base, int64_t item_stride, int64_t items, cudaStream_t st) {
  return launch_merge_t(m, base, item_stride, items, st);
}

cudaError_t launch_merge(const MergeParams &m, float2 *base, int64_t item_stride, int64_t items, cudaStream_t st) {
  return launch_merge_t(m, base, item_stride, items, st);
}

cudaError_t launch_to_c64(const double2 *src, float2 *dst, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  to_c64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dst, n);
  tn_count_launch(1);
  return cudaGetLastError();
}

cudaError_t launch_pack_bits(const uint64_t *src, uint64_t *dst, int64_t n_words, cudaStream_t st) {
  if (n_words <= 0) return cudaSuccess;
  copy_words_kernel<<<(unsigned)((n_words + 255) / 256), 256, 0, st>>>(src, dst, n_words);
  tn_count_launch(1);
  return cudaGetLastError();
}

"""The tensor-network-states amplitude method, step by step (oracle; test
infrastructure only).

Plain complex128 NumPy, LAPACK SVD via ``numpy.linalg.svd``. Every function
names the equation of the paper it follows. Nothing here is blocked, fused or
reordered beyond what those equations state; it is meant to be checked
against the paper by eye.

Conventions (readings where the paper is silent):

* Node tensor A^q has axis 0 = physical index sigma_q and then one auxiliary
  axis per incident edge, in increasing edge id (Eq. initialstate).
* A two-qubit gate matrix m is indexed [(s_k' s_l'), (s_k s_l)] with k = q[0]
  the high bit. After the gate the auxiliary index of the shared edge becomes
  the pair (a, s) with combined index a * chi_o + s on both endpoints
  (Eqs. result1/result2).
* Compression SVDs one endpoint (Eqs. svd/svd2 leave the choice open: "say
  A^k"). The endpoint is fixed by the circuit structure alone, never by the
  data: in the structural shapes (every bond starts at 1; a gate with chi_o
  terms multiplies its bond by chi_o; the compression bounds it by the row
  count of the SVD'd matrix and by chi) it is the endpoint whose matrix has
  fewer rows 2 * prod(other legs), ties to q[0]. With truncation, which
  endpoint is compressed changes the result, so a data-independent rule is
  what makes the result well defined for every bitstring. The compression keeps
  singular values > cutoff * s_0, at most chi (chi = 0: no cap), and never
  renormalises.
* The bra half starts from the product vector |s> and applies the transposes
  of the second group of gates from the last one back to the first; the
  amplitude is then sum_sigma psi_bar[sigma] phi[sigma] with no complex
  conjugation (Eq. overlap). This equals applying the group "inversely" to
  <s| (Fig. 2a).
* ``compress="two_sided"`` selects a variant of Eqs. svd/svd2 that the paper does not use: thin QR
  of both endpoints, SVD of the small bond matrix R_k R_l^T, isometry to the same endpoint and
  S to the other. It keeps the singular values of the local product A^k A^l itself, so its
  truncation is the best one of that rank for the pair (Eckart-Young) and its bond is the rank of
  the product. Same keep rule and endpoint rule; untruncated it gives the same amplitudes.
* Single-qubit gates are applied to the physical index directly (no fusion).
* Overlap legs merge (a, b) as a * dim(b) + b (Eq. overlap).
* Cutting fixes the merged index of the cut edges; the slices' scalars are
  summed (overlap paragraph: cutting).
* The contraction uses the oracle's own greedy pairwise order (smallest
  result first); the result does not depend on the order.
"""
from __future__ import annotations

import itertools
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np


# --------------------------------------------------------------------------
# Eq. gatesplit
# --------------------------------------------------------------------------
def gate_split(m: np.ndarray, rel: float = 1e-12):
    """Split a 4x4 gate O into P[s_k', s_k, s] and Q[s_l', s_l, s] (Eq. gatesplit).

    O is regrouped as a matrix with rows (s_k', s_k) and columns (s_l', s_l)
    and factorised by SVD; chi_o = number of singular values above
    ``rel * s_0``; the singular values are split evenly (sqrt) between P and Q.
    """
    O4 = np.asarray(m, dtype=np.complex128).reshape(2, 2, 2, 2)       # [k', l', k, l]
    R = O4.transpose(0, 2, 1, 3).reshape(4, 4)                          # [(k',k), (l',l)]
    U, S, Vh = np.linalg.svd(R)
    chi_o = int(np.sum(S > rel * S[0]))
    sq = np.sqrt(S[:chi_o])
    P = (U[:, :chi_o] * sq[None, :]).reshape(2, 2, chi_o)
    Q = (sq[:, None] * Vh[:chi_o, :]).T.reshape(2, 2, chi_o)
    return P, Q, chi_o


# --------------------------------------------------------------------------
# the state
# --------------------------------------------------------------------------
class TNS:
    """A tensor network state on a qubit graph (Eq. initialstate)."""

    def __init__(self, n: int, edges: Sequence[Tuple[int, int]], bits: Optional[Sequence[int]] = None):
        self.n = n
        self.edges = [tuple(sorted(e)) for e in edges]
        self.edge_id: Dict[Tuple[int, int], int] = {e: i for i, e in enumerate(self.edges)}
        self.legs: List[List[int]] = [[] for _ in range(n)]
        for i, (u, v) in enumerate(self.edges):
            self.legs[u].append(i)
            self.legs[v].append(i)
        self.A: List[np.ndarray] = []
        for q in range(n):
            t = np.zeros((2,) + (1,) * len(self.legs[q]), dtype=np.complex128)
            t[int(bits[q]) if bits is not None else 0] = 1.0
            self.A.append(t)
        self.log: List[dict] = []     # one record per compression

    def bond(self, e: int) -> int:
        u = self.edges[e][0]
        return self.A[u].shape[1 + self.legs[u].index(e)]

    def bonds(self) -> List[int]:
        return [self.bond(e) for e in range(len(self.edges))]

    # Eqs. result1 / result2 (and a plain single-qubit application)
    def apply_1q(self, q: int, u: np.ndarray) -> None:
        self.A[q] = np.tensordot(np.asarray(u, dtype=np.complex128), self.A[q], axes=(1, 0))

    @staticmethod
    def _apply_half(T: np.ndarray, P: np.ndarray, pos: int) -> np.ndarray:
        """A[s', ..., (a s), ...] = sum_sigma P[s', sigma, s] A[sigma, ..., a, ...]."""
        out = np.tensordot(P, T, axes=(1, 0))          # [s', s, legs...]
        out = np.moveaxis(out, 1, pos + 1)             # s right after leg ``pos``
        shape = list(T.shape)
        shape[pos] *= P.shape[2]
        return out.reshape(shape)

    def apply_2q(self, q0: int, q1: int, m: np.ndarray, chi: int = 0, cutoff: float = 1e-12,
                 svd_node: Optional[int] = None, compress: str = "one_sided") -> None:
        """Eqs. result1/result2, then the bond compression: Eqs. svd/svd2 (``one_sided``) or the
        two-sided variant (``two_sided``, see ``_compress_two_sided``)."""
        k, l = q0, q1
        e = self.edge_id.get(tuple(sorted((k, l))))
        if e is None:
            raise ValueError(f"gate on non-edge ({k},{l})")
        P, Q, chi_o = gate_split(m)
        pk = 1 + self.legs[k].index(e)
        pl = 1 + self.legs[l].index(e)
        Ak = self._apply_half(self.A[k], P, pk)
        Al = self._apply_half(self.A[l], Q, pl)
        # Eqs. svd / svd2: SVD one endpoint, absorb S V into the other
        rows_k = Ak.size // Ak.shape[pk]
        rows_l = Al.size // Al.shape[pl]
        if (rows_k <= rows_l) if svd_node is None else (svd_node == k):
            Asv, psv, Aot, pot, sv = Ak, pk, Al, pl, k
        else:
            Asv, psv, Aot, pot, sv = Al, pl, Ak, pk, l
        if compress == "two_sided":
            Asv, Aot = self._compress_two_sided(Asv, psv, Aot, pot, chi, cutoff, e, sv)
            if sv == k:
                self.A[k], self.A[l] = Asv, Aot
            else:
                self.A[k], self.A[l] = Aot, Asv
            return
        if compress != "one_sided":
            raise ValueError(f"unknown compression {compress!r}")
        X = np.moveaxis(Asv, psv, -1)
        shp = X.shape
        X = X.reshape(-1, shp[-1])
        U, S, Vh = np.linalg.svd(X, full_matrices=False)
        keep = int(np.sum(S > cutoff * S[0])) if S[0] > 0 else 1
        if chi and chi > 0:
            keep = min(keep, chi)
        keep = max(keep, 1)
        Asv = np.moveaxis(U[:, :keep].reshape(shp[:-1] + (keep,)), -1, psv)
        Vp = S[:keep, None] * Vh[:keep, :]
        Aot = np.moveaxis(np.tensordot(Aot, Vp, axes=(pot, 1)), -1, pot)
        if sv == k:
            self.A[k], self.A[l] = Asv, Aot
        else:
            self.A[k], self.A[l] = Aot, Asv
        self.log.append(dict(edge=e, svd_node=sv, m=X.shape[0], n=X.shape[1], s=S, keep=keep))

    def _compress_two_sided(self, Asv, psv, Aot, pot, chi, cutoff, e, sv):
        """Two-sided bond compression, a variant of Eqs. svd/svd2 that the paper does not use.

        With X = A^sv and Y = A^other matricised as (physical and other legs) x (bond), the two
        tensors meet in the local product X Y^T. Thin QR factorisations X = Q_x R_x and
        Y = Q_y R_y reduce it to the small bond matrix R_x R_y^T, whose SVD U S V^H has the
        singular values of X Y^T itself (Q_x, Q_y have orthonormal columns). The kept part gives
        A^sv <- Q_x U (an isometry, as in Eq. svd2) and A^other <- Q_y conj(V) S, so
        X' Y'^T = Q_x U S V^H Q_y^T: the best approximation of X Y^T of that rank (Eckart-Young),
        and a bond no larger than the rank of X Y^T. Same keep rule as the one-sided form."""
        X = np.moveaxis(Asv, psv, -1)
        shx = X.shape
        X = X.reshape(-1, shx[-1])
        Y = np.moveaxis(Aot, pot, -1)
        shy = Y.shape
        Y = Y.reshape(-1, shy[-1])
        Qx, Rx = np.linalg.qr(X)
        Qy, Ry = np.linalg.qr(Y)
        Mb = Rx @ Ry.T
        U, S, Vh = np.linalg.svd(Mb, full_matrices=False)
        keep = int(np.sum(S > cutoff * S[0])) if S[0] > 0 else 1
        if chi and chi > 0:
            keep = min(keep, chi)
        keep = max(keep, 1)
        Xn = Qx @ U[:, :keep]
        Yn = Qy @ (S[:keep, None] * Vh[:keep, :]).T
        self.log.append(dict(edge=e, svd_node=sv, m=Mb.shape[0], n=Mb.shape[1], s=S, keep=keep,
                             two_sided=True))
        return (np.moveaxis(Xn.reshape(shx[:-1] + (keep,)), -1, psv),
                np.moveaxis(Yn.reshape(shy[:-1] + (keep,)), -1, pot))

    def apply(self, gate, chi: int = 0, cutoff: float = 1e-12, transpose: bool = False,
              svd_node: Optional[int] = None, compress: str = "one_sided") -> None:
        m = gate.m.T if transpose else gate.m
        if len(gate.qubits) == 1:
            self.apply_1q(gate.qubits[0], m)
        else:
            self.apply_2q(gate.qubits[0], gate.qubits[1], m, chi, cutoff, svd_node, compress)


def structural_svd_nodes(n, edges, gates, chi=0, return_dims: bool = False):
    """The endpoint each two-qubit gate of ``gates`` (in application order) compresses: the one
    whose matrix has fewer rows 2 * prod(other legs) in the structural shapes, ties to the gate's
    first qubit. Structural shapes: bonds start at 1; a gate multiplies its bond by its chi_o
    (Eq. gatesplit); the compression bounds it by the rows of the compressed matrix and by chi
    (Eqs. svd, shouwei). The same shapes bound the two-sided compression: the rank of the local
    product is at most the smaller endpoint's rows, which is the endpoint named here. Independent
    of the state."""
    es = [tuple(sorted(e)) for e in edges]
    eid = {e: i for i, e in enumerate(es)}
    legs: List[List[int]] = [[] for _ in range(n)]
    for i, (u, v) in enumerate(es):
        legs[u].append(i)
        legs[v].append(i)
    d = [1] * len(es)
    out = []
    for g in gates:
        if len(g.qubits) == 1:
            continue
        k, l = g.qubits
        e = eid[tuple(sorted((k, l)))]
        chi_o = gate_split(g.m)[2]
        rows_k = 2 * math.prod(d[f] for f in legs[k] if f != e)
        rows_l = 2 * math.prod(d[f] for f in legs[l] if f != e)
        node, rows = (k, rows_k) if rows_k <= rows_l else (l, rows_l)
        nd = min(d[e] * chi_o, rows)
        if chi and chi > 0:
            nd = min(nd, chi)
        d[e] = nd
        out.append(node)
    return (out, d) if return_dims else out


# --------------------------------------------------------------------------
# two-sided evolution (Fig. 2a)
# --------------------------------------------------------------------------
def split_gates(gates, split_cycle: int):
    g1 = [g for g in gates if g.cycle <= split_cycle]
    g2 = [g for g in gates if g.cycle > split_cycle]
    return g1, g2


def _evolve(t: TNS, seq, chi, cutoff, transpose, compress="one_sided") -> TNS:
    nodes = iter(structural_svd_nodes(t.n, t.edges, seq, chi))
    for g in seq:
        t.apply(g, chi, cutoff, transpose=transpose,
                svd_node=None if len(g.qubits) == 1 else next(nodes), compress=compress)
    return t


def evolve_ket(n, edges, gates1, chi=0, cutoff=1e-12, compress="one_sided") -> TNS:
    """|phi> = (group 1) |0...0>."""
    return _evolve(TNS(n, edges), list(gates1), chi, cutoff, False, compress)


def evolve_bra(n, edges, gates2, bits, chi=0, cutoff=1e-12, compress="one_sided") -> TNS:
    """Coefficients of <psi| = <s| (group 2): the transposed gates, last to first, on |s>."""
    return _evolve(TNS(n, edges, bits), list(reversed(list(gates2))), chi, cutoff, True, compress)


# --------------------------------------------------------------------------
# Eq. overlap, cutting and contraction
# --------------------------------------------------------------------------
def overlap_node(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """C[..., (a_e b_e), ...] = sum_sigma A[sigma, ..., a_e, ...] B[sigma, ..., b_e, ...]."""
    r = A.ndim - 1
    sub_a = [0] + [1 + j for j in range(r)]
    sub_b = [0] + [1 + r + j for j in range(r)]
    sub_c = [x for j in range(r) for x in (1 + j, 1 + r + j)]
    C = np.einsum(A, sub_a, B, sub_b, sub_c)
    shape = [A.shape[1 + j] * B.shape[1 + j] for j in range(r)]
    return C.reshape(shape)


def contract_network(tensors: List[np.ndarray], labels: List[List[int]]) -> complex:
    """Contract a closed network; edge labels appear on exactly two tensors.

    Order: repeatedly contract the pair of tensors sharing a label whose result
    has the fewest elements (ties: lowest indices); disconnected pieces are
    multiplied at the end.
    """
    ts = list(tensors)
    ls = [list(l) for l in labels]
    while len(ts) > 1:
        best = None
        for i in range(len(ts)):
            si = set(ls[i])
            for j in range(i + 1, len(ts)):
                shared = si.intersection(ls[j])
                if not shared:
                    continue
                size = 1
                for a, lab in enumerate(ls[i]):
                    if lab not in shared:
                        size *= ts[i].shape[a]
                for a, lab in enumerate(ls[j]):
                    if lab not in shared:
                        size *= ts[j].shape[a]
                if best is None or size < best[0]:
                    best = (size, i, j, shared)
        if best is None:                        # no shared labels left: scalars / products
            i, j, shared = 0, 1, set()
        else:
            _, i, j, shared = best
        shared = sorted(shared)
        ai = [ls[i].index(x) for x in shared]
        aj = [ls[j].index(x) for x in shared]
        t = np.tensordot(ts[i], ts[j], axes=(ai, aj))
        lab = [x for x in ls[i] if x not in shared] + [x for x in ls[j] if x not in shared]
        for idx in sorted((i, j), reverse=True):
            del ts[idx]
            del ls[idx]
        ts.append(t)
        ls.append(lab)
    return complex(ts[0].reshape(()) if ts[0].ndim == 0 else ts[0].sum())


def double_layer_amplitude(ket: TNS, bra: TNS) -> complex:
    """<psi|phi> from the double-layer network: every ket tensor A^q and every bra tensor B^q is a
    node of its own, A^q and B^q share the physical index sigma_q, the A's share the ket bonds
    and the B's the bra bonds. These are the sums of Eq. overlap without first forming the node
    tensors C^q = sum_sigma A^q B^q, so the value equals overlap_amplitude; only the grouping of
    the sums differs (here: the oracle's greedy pairwise order over 2N tensors)."""
    ts, ls = [], []
    for q in range(ket.n):
        ts.append(ket.A[q])
        ls.append([("s", q)] + [("a", e) for e in ket.legs[q]])
        ts.append(bra.A[q])
        ls.append([("s", q)] + [("b", e) for e in bra.legs[q]])
    return contract_network(ts, ls)


def overlap_amplitude(ket: TNS, bra: TNS, cuts: Sequence[int] = (), slices=None) -> complex:
    """<psi|phi> by Eq. overlap; with ``cuts`` the sum over all slices of the cut edges.

    ``slices``: if given, only the slices with these indices enter the sum (index = position in
    the enumeration of the cut edges' values, first cut edge most significant; with no cuts the
    one slice is index 0)."""
    C = [overlap_node(ket.A[q], bra.A[q]) for q in range(ket.n)]
    labels = [list(ket.legs[q]) for q in range(ket.n)]
    cuts = list(cuts)
    if not cuts:
        if slices is not None and 0 not in slices:
            return 0j
        return contract_network(C, labels)
    dims = [C[ket.edges[e][0]].shape[labels[ket.edges[e][0]].index(e)] for e in cuts]
    total = 0j
    for k, vals in enumerate(itertools.product(*[range(d) for d in dims])):
        if slices is not None and k not in slices:
            continue
        sub, sl = [], []
        for q in range(ket.n):
            t, lab = C[q], labels[q]
            idx = [slice(None)] * t.ndim
            keep = []
            for a, x in enumerate(lab):
                if x in cuts:
                    idx[a] = vals[cuts.index(x)]
                else:
                    keep.append(x)
            sub.append(t[tuple(idx)])
            sl.append(keep)
        total += contract_network(sub, sl)
    return total


def to_dense(t: TNS) -> np.ndarray:
    """The full coefficient array (shape (2,)*N, axis q = qubit q) of a small TNS:
    F(A^1 ... A^N) of Eq. initialstate with every physical index left open."""
    ts, ls = [], []
    for q in range(t.n):
        ts.append(t.A[q])
        ls.append([("p", q)] + list(t.legs[q]))
    out, lab = ts[0], ls[0]
    for q in range(1, t.n):
        shared = [x for x in lab if x in ls[q]]
        out = np.tensordot(out, ts[q], axes=([lab.index(x) for x in shared], [ls[q].index(x) for x in shared]))
        lab = [x for x in lab if x not in shared] + [x for x in ls[q] if x not in shared]
    return np.transpose(out, [lab.index(("p", q)) for q in range(t.n)])


def amplitudes(n, edges, gates, bits_batch, split_cycle, chi=0, cutoff=1e-12, cuts=(), ket=None, slices=None,
               compress="one_sided"):
    """The full method for each row of ``bits_batch``; returns (amplitudes, ket). ``slices``: only
    these slices of the cut network enter each sum (see overlap_amplitude). ``compress``: the bond
    compression of both halves, ``one_sided`` (Eqs. svd/svd2) or ``two_sided``."""
    g1, g2 = split_gates(gates, split_cycle)
    if ket is None:
        ket = evolve_ket(n, edges, g1, chi, cutoff, compress)
    out = np.empty(len(bits_batch), dtype=np.complex128)
    for i, bits in enumerate(bits_batch):
        bra = evolve_bra(n, edges, g2, bits, chi, cutoff, compress)
        out[i] = overlap_amplitude(ket, bra, cuts, slices)
    return out, ket

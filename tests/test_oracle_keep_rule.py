"""The one-sided keep rule of the oracle's bond compression (Eqs. svd/svd2) against what the
mathematics fixes, with planted mistakes that must fail.

The compression of Eqs. svd/svd2 takes the SVD X = U S V^H of the compressed endpoint matricised
as (physical and other legs) x (bond), keeps the singular values above cutoff * s_0, at most chi,
largest first, and replaces the pair (X, Y) by (U_k, Y (S_k V_k^H)^T). The product of the pair
over the bond is then X_k Y^T with X_k = U_k S_k V_k^H, the best rank-k approximation of X
(Eckart-Young). Here X is built from factors chosen in the test (known singular values), so the
expected product, the kept rank and the lost weight follow from those factors alone."""
import numpy as np
import pytest
import scipy.linalg

import gen
from oracle import tns

# known spectrum of the compressed endpoint (distinct, s_0 far from 1 so that a cutoff read as
# absolute keeps a different count than one read relative to s_0)
S_KNOWN = np.array([40.0, 24.0, 12.0, 6.0, 0.8, 0.02])
D0, D1 = 6, 4          # bond being compressed (qubit 0 -- qubit 1), other leg of qubit 1 (to qubit 2)


def _haar_isometry(g, m, n):
    z = g.standard_normal((m, n)) + 1j * g.standard_normal((m, n))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


def _chain_with_known_endpoint(seed=3):
    """A 3-qubit chain 0 - 1 - 2 (edges e0 = (0, 1), e1 = (1, 2)) whose middle tensor, matricised
    as (sigma_1, leg e1) x (leg e0), is X = U diag(S_KNOWN) V^H with Haar U, V. Returns the state,
    X and its factors."""
    g = np.random.default_rng(seed)
    t = tns.TNS(3, [(0, 1), (1, 2)])
    U = _haar_isometry(g, 2 * D1, D0)
    V = _haar_isometry(g, D0, D0)
    X = U @ np.diag(S_KNOWN) @ V.conj().T                           # rows (sigma_1, d1), cols b0
    t.A[1] = X.reshape(2, D1, D0).transpose(0, 2, 1).copy()          # [sigma_1, e0, e1]
    t.A[0] = g.standard_normal((2, D0)) + 1j * g.standard_normal((2, D0))
    t.A[2] = g.standard_normal((2, D1)) + 1j * g.standard_normal((2, D1))
    return t, X, U, V


def _pair_product(t):
    """Qubits 0 and 1 contracted over e0: [sigma_0, sigma_1, d1]."""
    return np.tensordot(t.A[0], t.A[1], axes=(1, 1))


def _expected_product(A0, U, V, keep):
    Xk = U[:, :keep] @ np.diag(S_KNOWN[:keep]) @ V[:, :keep].conj().T
    return np.tensordot(A0, Xk.reshape(2, D1, D0), axes=(1, 2))     # [sigma_0, sigma_1, d1]


def _compress(t, chi, cutoff):
    """The identity gate on (0, 1) (one term, so the bond keeps its D0 values), node 1 compressed."""
    t.apply_2q(0, 1, np.eye(4), chi=chi, cutoff=cutoff, svd_node=1)


# (chi, cutoff, kept): the cap binds; the cutoff binds (relative: s > 4.0 keeps 40, 24, 12, 6);
# both given and the cutoff binds; both given and the cap binds; nothing truncated
CASES = [(2, 1e-12, 2), (0, 0.1, 4), (5, 0.1, 4), (3, 1e-3, 3), (0, 1e-12, 6)]


@pytest.mark.parametrize("chi,cutoff,kept", CASES)
def test_one_sided_compression_is_the_rank_k_truncation_of_the_endpoint(chi, cutoff, kept):
    t, X, U, V = _chain_with_known_endpoint()
    A0 = t.A[0].copy()
    _compress(t, chi, cutoff)
    assert t.bond(0) == kept
    ref = _expected_product(A0, U, V, kept)
    got = _pair_product(t)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # the compressed endpoint is an isometry (Eq. svd2: A^k <- U), the untouched qubit 2 as before
    M1 = np.moveaxis(t.A[1], 1, -1).reshape(-1, kept)
    assert np.allclose(M1.conj().T @ M1, np.eye(kept), atol=1e-12)
    # lost weight of the endpoint: ||X - X_k||_F^2 = sum of the dropped s^2 (no renormalisation)
    X_after = U[:, :kept] @ np.diag(S_KNOWN[:kept]) @ V[:, :kept].conj().T
    assert abs(np.linalg.norm(X - X_after) ** 2 - np.sum(S_KNOWN[kept:] ** 2)) < 1e-9


def test_kept_values_are_the_largest_of_the_matricised_endpoint_on_a_haar_grid(monkeypatch):
    """On a generic Haar 3x4 grid circuit capped at chi = 3, after every compression the compressed
    endpoint spans the left singular subspace of the chi largest singular values of the matrix
    that was decomposed, as an independent SVD routine (scipy's LAPACK gesvd driver) finds it.
    The matrix is taken where the oracle hands it to numpy's SVD (the calls with
    full_matrices=False are the compressions; the gate split uses full matrices)."""
    g = gen.grid(3, 4)
    gates = gen.rqc(g, 4, gen.rng(21, 1), twoq="haar", oneq="haar")
    chi = 3
    decomposed = []
    np_svd = np.linalg.svd

    def spy(a, full_matrices=True, **kw):
        if not full_matrices:
            decomposed.append(np.array(a, copy=True))
        return np_svd(a, full_matrices=full_matrices, **kw)

    orig = tns.TNS.apply_2q
    truncating = [0]

    def checked(self, q0, q1, m, chi=0, cutoff=1e-12, svd_node=None, compress="one_sided"):
        orig(self, q0, q1, m, chi, cutoff, svd_node, compress)
        rec, X = self.log[-1], decomposed[-1]
        kept = rec["keep"]
        Uq, Sq, _ = scipy.linalg.svd(X, full_matrices=False, lapack_driver="gesvd")
        rank = int(np.sum(Sq > 1e-12 * Sq[0]))
        assert kept == min(rank, chi)
        if kept < rank:
            truncating[0] += 1
            assert Sq[kept - 1] > (1 + 1e-6) * Sq[kept]      # a gap: the kept subspace is unique
        e, sv_n = rec["edge"], rec["svd_node"]
        Ms = np.moveaxis(self.A[sv_n], 1 + self.legs[sv_n].index(e), -1).reshape(-1, kept)
        P = Uq[:, :kept] @ Uq[:, :kept].conj().T
        assert np.allclose(Ms @ Ms.conj().T, P, atol=1e-10)

    monkeypatch.setattr(np.linalg, "svd", spy)
    monkeypatch.setattr(tns.TNS, "apply_2q", checked)
    tns.evolve_ket(12, g.edges, gates, chi=chi, cutoff=1e-12)
    assert truncating[0] >= 5


# -- planted mistakes (on the CPU): each must fail the hand-built pin above -------------------

def _planted_one_sided(monkeypatch, mistake):
    orig = tns.TNS.apply_2q

    def faulty(self, q0, q1, m, chi=0, cutoff=1e-12, svd_node=None, compress="one_sided"):
        k, l = q0, q1
        e = self.edge_id[tuple(sorted((k, l)))]
        P, Q, chi_o = tns.gate_split(m)
        pk, pl = 1 + self.legs[k].index(e), 1 + self.legs[l].index(e)
        Ak, Al = self._apply_half(self.A[k], P, pk), self._apply_half(self.A[l], Q, pl)
        sv_n = svd_node if svd_node is not None else (k if Ak.size // Ak.shape[pk] <= Al.size // Al.shape[pl] else l)
        Asv, psv, Aot, pot = (Ak, pk, Al, pl) if sv_n == k else (Al, pl, Ak, pk)
        X = np.moveaxis(Asv, psv, -1)
        shp = X.shape
        X = X.reshape(-1, shp[-1])
        U, S, Vh = np.linalg.svd(X, full_matrices=False)
        if mistake == "keep_smallest":
            U, S, Vh = U[:, ::-1], S[::-1], Vh[::-1, :]
        thr = cutoff if mistake == "absolute_cutoff" else cutoff * S.max()
        keep = int(np.sum(S > thr))
        if chi:
            keep = min(keep, chi)
        Sk = S[:keep]
        if mistake == "renormalise":
            Sk = Sk * np.sqrt(np.sum(S ** 2) / np.sum(Sk ** 2))
        Asv = np.moveaxis(U[:, :keep].reshape(shp[:-1] + (keep,)), -1, psv)
        Vp = Sk[:, None] * Vh[:keep, :]
        Aot = np.moveaxis(np.tensordot(Aot, Vp, axes=(pot, 1)), -1, pot)
        if sv_n == k:
            self.A[k], self.A[l] = Asv, Aot
        else:
            self.A[k], self.A[l] = Aot, Asv
        self.log.append(dict(edge=e, svd_node=sv_n, m=X.shape[0], n=X.shape[1], s=S, keep=keep))
    monkeypatch.setattr(tns.TNS, "apply_2q", faulty)
    return orig


def _pin_holds(chi, cutoff, kept):
    t, X, U, V = _chain_with_known_endpoint()
    A0 = t.A[0].copy()
    _compress(t, chi, cutoff)
    if t.bond(0) != kept:
        return False
    ref = _expected_product(A0, U, V, kept)
    return bool(np.max(np.abs(_pair_product(t) - ref)) <= 1e-12 * np.max(np.abs(ref)))


def test_faithful_restatement_passes_the_pin(monkeypatch):
    _planted_one_sided(monkeypatch, "none")
    assert all(_pin_holds(*c) for c in CASES)


@pytest.mark.parametrize("mistake", ["keep_smallest", "absolute_cutoff", "renormalise"])
def test_planted_keep_rule_mistakes_are_caught(monkeypatch, mistake):
    _planted_one_sided(monkeypatch, mistake)
    assert not all(_pin_holds(*c) for c in CASES)

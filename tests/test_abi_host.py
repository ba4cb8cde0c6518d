"""C-ABI library on the CPU: it loads, exports every entry point declared in
include/tn.h, and its host-only pieces (gate split, Algorithm 1, input
validation) agree with the oracle and the paper. No device compute here."""
import math
import os
import re

import numpy as np
import pytest

import gen
from oracle import path as opath
from oracle import tns as otns


@pytest.fixture(scope="module")
def tn(repo_root):
    from paper_2011_02621_gb300 import build
    build.build()
    from paper_2011_02621_gb300 import tn as _tn
    return _tn


def declared_symbols(repo_root):
    txt = open(os.path.join(repo_root, "include", "tn.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(tn, repo_root):
    names = declared_symbols(repo_root)
    assert len(names) >= 15
    for name in names:
        assert hasattr(tn.LIB, name), name


def test_gate_split_matches_oracle_and_reconstructs(tn):
    rng = gen.rng(5, 1)
    for m in (gen.fsim(math.pi / 2, math.pi / 6), gen.fsim(0, math.pi), gen.haar_u4(rng), np.eye(4, dtype=complex)):
        P, Q, chi = tn.tn_gate_split(m)
        _, _, chi_o = otns.gate_split(m)
        assert chi == chi_o
        rec = np.einsum("aks,bls->abkl", P, Q).reshape(4, 4)
        assert np.max(np.abs(rec - m)) < 1e-13


def random_graph(n, rng):
    edges = set()
    for i in range(1, n):
        edges.add((int(rng.integers(i)), i))
    for _ in range(n):
        u, v = sorted(rng.choice(n, 2, replace=False))
        edges.add((int(u), int(v)))
    return sorted(edges)


def test_algorithm1_unconstrained_is_global_optimum(tn):
    """Eq. optscore: without Assumptions 1-3 Algorithm 1 is a subset Dijkstra and finds the optimum."""
    rng = np.random.default_rng(11)
    for n in (4, 5, 6, 7, 8):
        for _ in range(3):
            edges = random_graph(n, rng)
            dims = rng.integers(2, 17, size=len(edges)).astype(float)
            order, score, _ = tn.tn_path_search(n, edges, dims, boundary_only=False, connected=False)
            assert sorted(order) == list(range(n))
            assert score == pytest.approx(opath.score(list(order), edges, dims), rel=1e-12)
            assert score == pytest.approx(opath.subset_dp_optimum(n, edges, dims), rel=1e-12)
            if n <= 7:
                assert score == pytest.approx(opath.bruteforce_optimum(n, edges, dims), rel=1e-12)


def test_algorithm1_with_assumptions_is_valid_and_not_below_optimum(tn):
    rng = np.random.default_rng(12)
    for n in (6, 7, 8, 9):
        edges = random_graph(n, rng)
        dims = rng.integers(2, 9, size=len(edges)).astype(float)
        order, score, _ = tn.tn_path_search(n, edges, dims)
        assert sorted(order) == list(range(n))
        assert score == pytest.approx(opath.score(list(order), edges, dims), rel=1e-12)
        assert score >= opath.subset_dp_optimum(n, edges, dims) * (1 - 1e-12)
        deg = np.zeros(n, int)
        for u, v in edges:
            deg[u] += 1
            deg[v] += 1
        if (deg < deg.max()).any():
            assert deg[order[0]] < deg.max()          # Assumption 1: start on the boundary


def test_algorithm1_partial_paths_almost_connected(tn):
    """Assumption 3: every prefix is connected, or connected plus one qubit that the next step reconnects."""
    g = gen.staggered(6, 9, remove_seed=gen.BASE_SEED + 3)
    dims = np.full(len(g.edges), 4.0)
    order, score, _ = tn.tn_path_search(g.n, g.edges, dims)
    adj = {q: set() for q in range(g.n)}
    for u, v in g.edges:
        adj[u].add(v)
        adj[v].add(u)
    seen = set()
    for m, q in enumerate(order):
        seen.add(int(q))
        comps, todo = 0, set(seen)
        while todo:
            comps += 1
            st = [todo.pop()]
            while st:
                x = st.pop()
                for y in adj[x]:
                    if y in todo:
                        todo.discard(y)
                        st.append(y)
        assert comps <= 2
        if comps == 2:
            nxt = int(order[m + 1])
            assert adj[nxt] & seen


def test_algorithm1_rank_bound(tn):
    """Assumption 2: with max_rank M no intermediate has more than M open legs."""
    g = gen.grid(4, 5)
    dims = np.full(len(g.edges), 3.0)
    for M in (5, 6):
        order, _, _ = tn.tn_path_search(g.n, g.edges, dims, max_rank=M)
        S = set()
        for q in order:
            S.add(int(q))
            open_legs = sum(1 for u, v in g.edges if (u in S) != (v in S))
            assert open_legs <= M
    with pytest.raises(tn.TNError) as ei:
        tn.tn_path_search(g.n, g.edges, dims, max_rank=2)
    assert ei.value.status == tn.TN_ERR_NO_PATH


def test_build_validates_graph_and_gates(tn):
    g = gen.grid(2, 2)
    ok = gen.rqc(g, 2, gen.rng(1, 1))
    c = tn.tn_build(g.n, g.edges, ok, allocator=None)
    assert c.ptr
    with pytest.raises(tn.TNError) as ei:                 # disconnected
        tn.tn_build(4, [(0, 1), (2, 3)], [], allocator=None)
    assert ei.value.status == tn.TN_ERR_GRAPH
    with pytest.raises(tn.TNError) as ei:                 # gate on a non-edge (diagonal of the square)
        tn.tn_build(g.n, g.edges, [gen.Gate(1, (0, 3), np.eye(4, dtype=complex))], allocator=None)
    assert ei.value.status == tn.TN_ERR_GRAPH
    with pytest.raises(tn.TNError) as ei:                 # qubit out of range
        tn.tn_build(g.n, g.edges, [gen.Gate(1, (7,), np.eye(2, dtype=complex))], allocator=None)
    assert ei.value.status == tn.TN_ERR_GRAPH
    with pytest.raises(tn.TNError) as ei:                 # duplicate edge
        tn.tn_build(3, [(0, 1), (1, 0), (1, 2)], [], allocator=None)
    assert ei.value.status == tn.TN_ERR_GRAPH
    with pytest.raises(tn.TNError) as ei:                 # cycle 0 is not a cycle
        tn.tn_build(g.n, g.edges, [gen.Gate(0, (0,), np.eye(2, dtype=complex))], allocator=None)
    assert ei.value.status == tn.TN_ERR_ARG


def test_call_order_is_checked(tn):
    g = gen.grid(2, 2)
    c = tn.tn_build(g.n, g.edges, gen.rqc(g, 2, gen.rng(1, 1)), allocator=None)
    with pytest.raises(tn.TNError) as ei:
        tn.tn_path(c)
    assert ei.value.status == tn.TN_ERR_STATE
    with pytest.raises(tn.TNError) as ei:
        tn.tn_circuit_bond_dims(c, 0)
    assert ei.value.status == tn.TN_ERR_STATE


def test_no_cpu_fallback_without_gpu(tn):
    """On a machine without a CUDA device the device entry points fail loudly."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    g = gen.grid(2, 2)
    c = tn.tn_build(g.n, g.edges, gen.rqc(g, 2, gen.rng(1, 1)), allocator=None)
    with pytest.raises(tn.TNError) as ei:
        tn.tn_evolve_two_sided(c, 1)
    assert ei.value.status == tn.TN_ERR_CUDA


def test_cut_search_respects_limit_and_reports_cost(tn):
    """Cutting: every intermediate of the cut network fits the limit; total = slices x path score."""
    import math
    g = gen.grid(4, 5)
    rng = np.random.default_rng(4)
    dims = rng.choice([4, 8, 16, 32, 64], size=len(g.edges)).astype(float)
    order0, score0, _ = tn.tn_path_search(g.n, g.edges, dims)
    for limit in (1 << 22, 1 << 18, 1 << 14):
        order, cuts, total = tn.tn_cut_search(g.n, g.edges, dims, max_intermediate=limit)
        d2 = dims.copy()
        d2[list(cuts)] = 1
        S = set()
        for q in order:
            S.add(int(q))
            assert math.prod(d2[e] for e, (u, v) in enumerate(g.edges) if (u in S) != (v in S)) <= limit
        slices = math.prod(dims[e] for e in cuts)
        assert total == pytest.approx(slices * opath.score(list(order), g.edges, d2), rel=1e-12)
        assert total >= score0 * (1 - 1e-12) or len(cuts) == 0
    order, cuts, total = tn.tn_cut_search(g.n, g.edges, dims, n_cuts=0)
    assert len(cuts) == 0 and total == pytest.approx(score0, rel=1e-12)
    order, cuts, total = tn.tn_cut_search(g.n, g.edges, dims, cut_edges=[3, 7])
    assert list(cuts) == [3, 7]


def _oracle_dims(name):
    w = gen.workload(name, n_bits=1)
    g1, g2 = otns.split_gates(w.gates, w.split)
    ket = otns.evolve_ket(w.graph.n, w.graph.edges, g1, w.chi, w.cutoff)
    bra = otns.evolve_bra(w.graph.n, w.graph.edges, g2, w.bits[0], w.chi, w.cutoff)
    return w, [ket.bond(e) for e in range(len(w.graph.edges))], [bra.bond(e) for e in range(len(w.graph.edges))]


def test_merge_search_groups_and_cost(tn):
    """Boundary-node merging on the 53-qubit workload's overlap network (the oracle's bond
    dimensions): every qubit belongs to one node, each node is a connected group of at most three
    qubits (physical index <= 8 values) named by one of its members, every node is in the
    contraction order once, and the merged network costs no more than the unmerged one."""
    w, kd, bd = _oracle_dims("syc53")
    n, edges = w.graph.n, w.graph.edges
    owner, order, n_cuts, cost = tn.tn_merge_search(n, edges, kd, bd)
    owner_u, order_u, _, cost_u = tn.tn_merge_search(n, edges, kd, bd, merge=False)
    assert list(owner_u) == list(range(n)) and len(order_u) == n
    reps = sorted(set(owner))
    assert len(reps) == len(order) < n and sorted(order) == reps
    adj = {q: set() for q in range(n)}
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    for r in reps:
        members = [q for q in range(n) if owner[q] == r]
        assert owner[r] == r and 1 <= len(members) <= 3
        seen, todo = {members[0]}, [members[0]]          # connected inside the group
        while todo:
            x = todo.pop()
            for y in adj[x]:
                if owner[y] == r and y not in seen:
                    seen.add(y)
                    todo.append(y)
        assert seen == set(members)
    assert n_cuts == 0 and cost <= cost_u * (1 + 1e-12)


def test_merge_search_leaf_and_kept_cut_edges(tn):
    """A path graph 0-1-2-3 with equal bonds: nodes are merged in index order while at least two
    remain (the leaf 0 into 1, then 2 into that node: physical index 8); an explicit cut edge is
    never merged away (its endpoints stay in different nodes)."""
    edges = [(0, 1), (1, 2), (2, 3)]
    owner, order, _, _ = tn.tn_merge_search(4, edges, [2, 2, 2], [2, 2, 2])
    assert list(owner) == [1, 1, 1, 3] and sorted(order) == [1, 3]
    owner, order, n_cuts, _ = tn.tn_merge_search(4, edges, [2, 2, 2], [2, 2, 2], cut_edges=[0])
    assert owner[0] != owner[1] and n_cuts == 1
    with pytest.raises(tn.TNError):
        tn.tn_merge_search(4, edges, [2, 0, 2], [2, 2, 2])


def test_planner_on_the_double_layer_network(tn):
    """Algorithm 1 on the double-layer network of the 53-qubit workload (ket and bra tensors as
    separate nodes, joined by a dimension-2 physical edge; structural bond dims): its cost is the
    oracle's path score of the order it returns, and about ten times below the cost of the
    overlap network (one node per qubit, edge dims dk * db) on the same bonds."""
    w = gen.workload("syc53", n_bits=1)
    n, edges = w.graph.n, [tuple(sorted(e)) for e in w.graph.edges]
    g1, g2 = otns.split_gates(w.gates, w.split)
    kd = otns.structural_svd_nodes(n, edges, g1, w.chi, return_dims=True)[1]
    bd = otns.structural_svd_nodes(n, edges, list(reversed(g2)), w.chi, return_dims=True)[1]
    _, cuts1, total1 = tn.tn_cut_search(n, edges, [a * b for a, b in zip(kd, bd)])
    e2 = edges + [(n + u, n + v) for u, v in edges] + [(q, n + q) for q in range(n)]
    d2 = [float(x) for x in list(kd) + list(bd) + [2] * n]
    order2, cuts2, total2 = tn.tn_cut_search(2 * n, e2, d2)
    assert len(cuts1) == 0 and len(cuts2) == 0
    assert sorted(int(v) for v in order2) == list(range(2 * n))
    assert total2 == pytest.approx(opath.score([int(v) for v in order2], e2, d2), rel=1e-12)
    assert total2 < 0.2 * total1


def _structural_dims(w, chi=None):
    n, edges = w.graph.n, [tuple(sorted(e)) for e in w.graph.edges]
    g1, g2 = otns.split_gates(w.gates, w.split)
    chi = w.chi if chi is None else chi
    kd = otns.structural_svd_nodes(n, edges, g1, chi, return_dims=True)[1]
    bd = otns.structural_svd_nodes(n, edges, list(reversed(g2)), chi, return_dims=True)[1]
    return n, edges, kd, bd


def _joined_steps(order, edges, dims, layer):
    """Joining partial paths restated from its definition (no cuts): walking the path, two
    consecutive nodes u, v of the same layer that share exactly one edge a are contracted with each
    other first and absorbed as one node when that lowers both the step's complex multiply-adds
    (the pair's own contraction counted for bra pairs, which are per bitstring) and the elements
    read and written, neither rising. Returns the (M, K, N) of the steps of the joined path and the
    pairs' own contraction costs (every pair, both layers)."""
    legs = {v: set() for v in range(len(layer))}
    for i, (u, v) in enumerate(edges):
        legs[u].add(i)
        legs[v].add(i)

    def D(S):
        return int(np.prod([dims[e] for e in S])) if S else 1

    order, O, j, pairs = list(order), set(), 0, []
    while j < len(order) - 1:
        u, v = order[j], order[j + 1]
        sh = legs[u] & legs[v]
        if layer[u] == layer[v] and len(sh) == 1:
            a = next(iter(sh))
            K1, N1, R1 = legs[u] & O, legs[u] - O, O - legs[u]
            O1 = R1 | N1
            K2, N2, R2 = legs[v] & O1, legs[v] - O1, O1 - legs[v]
            first = j == 0
            seq_mac = (0 if first else D(R1) * D(K1) * D(N1)) + D(R2) * D(K2) * D(N2)
            seq_el = (0 if first else D(R1) * (D(K1) + D(N1))) + D(R2) * (D(K2) + D(N2))
            Lw = (legs[u] | legs[v]) - {a}
            Kw, Nw, Rw = Lw & O, Lw - O, O - Lw
            pair = D(legs[u] | legs[v])
            w_mac = (0 if first else D(Rw) * D(Kw) * D(Nw)) + (pair if layer[u] == 2 else 0)
            w_el = 0 if first else D(Rw) * (D(Kw) + D(Nw))
            if w_mac <= seq_mac and w_el <= seq_el and (w_mac < seq_mac or w_el < seq_el):
                pairs.append(pair)
                legs[u], legs[v] = Lw, set()
                order.pop(j + 1)
                continue
        L = legs[order[j]]
        O = (O - L) | (L - O)
        j += 1
    O, steps = set(), []
    for u in order:
        L = legs[u]
        K, N, R = L & O, L - O, O - L
        steps.append((D(R), D(K), D(N)))
        O = R | N
    return steps, pairs


def test_joined_paths_beat_the_best_main_path(tn):
    """Joining partial paths (the relaxation of Assumption 3 in the supplement) on the double-layer
    network of a 2x4 grid circuit: the joined plan costs fewer complex multiply-adds per amplitude,
    every pair's own contraction counted in full, than the best single main path over all orders
    (Eq. optscore, the oracle's subset recursion), which is what Algorithm 1 finds unconstrained.
    The library's joined plan has the steps of the join restated on its order."""
    g = gen.grid(2, 4)
    n = g.n
    gates = gen.rqc(g, 4, gen.rng(3, 1))
    w = gen.Workload("g8", g, gates, 4, 2, 0, 1e-12, gen.bitstrings(n, 1, gen.rng(3, 2)))
    _, edges, kd, bd = _structural_dims(w)
    e2 = edges + [(n + u, n + v) for u, v in edges] + [(q, n + q) for q in range(n)]
    d2 = [int(x) for x in list(kd) + list(bd)] + [2] * n
    order, cuts, plain = tn.tn_cut_search(2 * n, e2, [float(x) for x in d2])
    assert len(cuts) == 0
    best_main = opath.subset_dp_optimum(2 * n, e2, d2)
    assert plain == best_main
    steps, pairs = _joined_steps([int(v) for v in order], e2, d2, [1] * n + [2] * n)
    total = sum(m * k * nn for m, k, nn in steps[1:]) + sum(pairs)
    assert pairs and total < best_main
    c = tn.tn_build(n, g.edges, gates, allocator=None)
    info = tn.tn_plan_estimate(c, 2, 0, 1e-12, layers=2)
    assert info["n_steps"] == len(steps) - 1
    assert info["cmacs"] == pytest.approx(sum(m * k * nn for m, k, nn in steps[1:]), rel=1e-12)


@pytest.mark.parametrize("name", ["grid12", "syc53"])
def test_plan_estimate_matches_the_oracle_structure(tn, name):
    """The host-only plan estimate (no device) builds the gate programs with the library's own
    structural recursion; its contraction cost equals the planner's cost on the oracle's
    structural bonds, for the merged overlap network, the unmerged one and the double-layer one,
    so both recursions give the same bonds. Every compiled table passed the plan's index check."""
    w = gen.workload(name, n_bits=1)
    n, edges, kd, bd = _structural_dims(w)
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates, allocator=None)
    merged = tn.tn_plan_estimate(c, w.split, w.chi, w.cutoff)
    owner, order, ncut, total = tn.tn_merge_search(n, edges, kd, bd)
    assert merged["n_nodes"] == len(order) and merged["n_steps"] == len(order) - 1
    assert merged["n_cuts"] == ncut == 0
    assert merged["cmacs"] == pytest.approx(total, rel=1e-12)
    flat = tn.tn_plan_estimate(c, w.split, w.chi, w.cutoff, merge=False)
    _, cuts1, total1 = tn.tn_cut_search(n, edges, [a * b for a, b in zip(kd, bd)])
    assert flat["n_nodes"] == n and flat["cmacs"] == pytest.approx(total1, rel=1e-12)
    dl = tn.tn_plan_estimate(c, w.split, w.chi, w.cutoff, layers=2, merge=False)
    e2 = edges + [(n + u, n + v) for u, v in edges] + [(q, n + q) for q in range(n)]
    d2 = [float(x) for x in list(kd) + list(bd) + [2] * n]
    order2, cuts2, total2 = tn.tn_cut_search(2 * n, e2, d2)
    assert dl["n_nodes"] == 2 * n and dl["n_steps"] == 2 * n - 1 and dl["n_cuts"] == len(cuts2)
    assert dl["cmacs"] == pytest.approx(total2, rel=1e-12)
    assert dl["cmacs"] < merged["cmacs"]
    # the joined double-layer plan (default): the steps of the join restated on the same order
    joined = tn.tn_plan_estimate(c, w.split, w.chi, w.cutoff, layers=2)
    steps, _ = _joined_steps([int(v) for v in order2], e2, [int(x) for x in d2], [1] * n + [2] * n)
    assert joined["n_steps"] == len(steps) - 1 < dl["n_steps"]
    assert joined["cmacs"] == pytest.approx(sum(m * k * nn for m, k, nn in steps[1:]), rel=1e-12)
    assert joined["bytes_c64"] == pytest.approx(sum(8 * (m * k + m * nn) for m, k, nn in steps[1:]), rel=1e-12)
    assert joined["cmacs"] < dl["cmacs"] and joined["bytes_c64"] < dl["bytes_c64"]


def test_double_layer_plans_with_cuts_and_every_split(tn):
    """Double-layer plans compile and pass the index check at every split of the 3x4 grid and
    with cuts forced by a small intermediate limit (slice tables of ket-only and bra-only nodes)."""
    w = gen.workload("grid12", n_bits=1)
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates, allocator=None)
    for split in range(0, w.depth + 1):
        info = tn.tn_plan_estimate(c, split, 0, 1e-12, layers=2, merge=False)
        assert info["n_steps"] == 2 * w.graph.n - 1
        joined = tn.tn_plan_estimate(c, split, 0, 1e-12, layers=2)
        assert joined["n_steps"] < info["n_steps"] and joined["cmacs"] <= info["cmacs"]
        assert joined["max_intermediate"] <= info["max_intermediate"]
    for merge in (False, True):
        cut = tn.tn_plan_estimate(c, 4, 0, 1e-12, layers=2, max_intermediate=64, merge=merge)
        assert cut["n_cuts"] > 0 and cut["n_slices"] > 1 and cut["max_intermediate"] <= 64
    with pytest.raises(tn.TNError) as e:
        tn.tn_plan_estimate(c, 4, 0, 1e-12, layers=2, cut_edges=[0])
    assert e.value.status == tn.TN_ERR_UNSUPPORTED
    with pytest.raises(tn.TNError) as e:
        tn.tn_plan_estimate(c, 4, 0, 1e-12, layers=3)
    assert e.value.status == tn.TN_ERR_ARG
    with pytest.raises(tn.TNError) as e:
        tn.tn_plan_estimate(c, -1, 0, 1e-12)
    assert e.value.status == tn.TN_ERR_ARG


def test_double_layer_network_of_the_104_qubit_grid(tn):
    """Algorithm 1's subset masks hold 256 nodes, so the double-layer network of the 104-qubit
    grid (208 nodes) is planned: the plan's cost equals the oracle's path score of the order the
    host-only search returns on the same structural bonds, and a graph of more than 256 nodes is
    refused with TN_ERR_UNSUPPORTED."""
    w = gen.workload("syc104", n_bits=1)
    n, edges, kd, bd = _structural_dims(w)
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates, allocator=None)
    dl = tn.tn_plan_estimate(c, w.split, w.chi, w.cutoff, layers=2, merge=False)
    e2 = edges + [(n + u, n + v) for u, v in edges] + [(q, n + q) for q in range(n)]
    d2 = [float(x) for x in list(kd) + list(bd) + [2] * n]
    order2, cuts2, total2 = tn.tn_cut_search(2 * n, e2, d2)
    assert tn.tn_plan_estimate(c, w.split, w.chi, w.cutoff, layers=2)["cmacs"] < dl["cmacs"]
    assert dl["n_nodes"] == 2 * n == 208 and dl["n_steps"] == 207 and dl["n_cuts"] == len(cuts2) == 0
    assert sorted(int(v) for v in order2) == list(range(2 * n))
    assert total2 == pytest.approx(opath.score([int(v) for v in order2], e2, d2), rel=1e-12)
    assert dl["cmacs"] == pytest.approx(total2, rel=1e-12)
    assert dl["cmacs"] < tn.tn_plan_estimate(c, w.split, w.chi, w.cutoff)["cmacs"]
    ring = [(i, (i + 1) % 257) for i in range(257)]
    with pytest.raises(tn.TNError) as e:
        tn.tn_path_search(257, ring, [2.0] * 257)
    assert e.value.status == tn.TN_ERR_UNSUPPORTED


def test_planning_failures_are_statuses_not_exceptions(tn):
    """Untruncated 12-cycle circuit on 40 qubits (random 3-regular graph): the overlap network
    needs about 1e9 slices, whose offset tables the plan cannot hold. The host-only call returns
    TN_ERR_UNSUPPORTED; no C++ exception (an allocation failure) crosses the C ABI."""
    w = gen.regular3_family(count=32, n_bits=1)[31]
    assert w.graph.n == 40
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates, allocator=None)
    with pytest.raises(tn.TNError) as e:
        tn.tn_plan_estimate(c, w.split, 0, 1e-12)
    assert e.value.status == tn.TN_ERR_UNSUPPORTED and "slices" in str(e.value)


@pytest.mark.parametrize("gib", [0.5, 2.0, 8.0])
def test_batch_size_fills_the_budget(tn, gib):
    """The plan's device batch is the largest number of bitstrings whose workspace (a fixed part,
    the merged ket, plus a part per bitstring) fits the budget: the reported workspace fits, one
    bitstring more would not (unless the 65536 cap binds), and the fixed part is counted once."""
    w = gen.workload("syc53", n_bits=1)
    c = tn.tn_build(w.graph.n, w.graph.edges, w.gates, allocator=None)
    budget = gib * 2 ** 30
    info = tn.tn_plan_estimate(c, w.split, w.chi, w.cutoff, layers=2, mem_budget_bytes=budget)
    ch, ws = info["chunk_bitstrings"], info["workspace_bytes"]
    assert 1 <= ch <= 65536 and ws <= budget
    small = tn.tn_plan_estimate(c, w.split, w.chi, w.cutoff, layers=2, mem_budget_bytes=2 ** 26)
    per = (ws - small["workspace_bytes"]) / (ch - small["chunk_bitstrings"])   # one bitstring's share
    fixed = ws - ch * per
    assert fixed > 0 and per > 0
    assert ch == 65536 or fixed + (ch + 1) * per > budget

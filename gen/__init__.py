"""Seeded synthetic inputs for the TNS amplitude method: qubit graphs, random
quantum circuits and output bitstrings.

This module is shared by the oracle, the tests and the benchmark. It holds no
arithmetic of the method itself (no gate splitting, no SVD, no contraction):
it only draws graphs, gate matrices and bitstrings from named, seeded numpy
PCG64 streams.

Workload shapes follow the problem statement of the paper (a connected qubit
graph whose edges carry the two-qubit gates, Eq. initialstate and the text
around it; random circuits of interlaced single-qubit layers and fSim layers
on Sycamore-like coupler patterns ABCDCDAB). The Sycamore layouts themselves
are not available, so seeded stand-ins of the same shape are generated here:

* ``grid(R, C)``: nearest-neighbour grid with patterns A/B (horizontal edges
  at even/odd column) and C/D (vertical edges at even/odd row).
* ``staggered(R, C)``: diagonal-coupled staggered grid, every qubit linked to at
  most 4 diagonal neighbours, patterns A/B (straight edges at even/odd row)
  and C/D (offset edges at even/odd row); optionally one seeded site removed.
* ``random_regular3(n)``: random 3-regular graph, edges coloured into layers.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

BASE_SEED = 2011_02621
SYCAMORE_SEQUENCE = "ABCDCDAB"


def rng(seed: int, stream: int) -> np.random.Generator:
    """Named PCG64 stream ``stream`` (0 graph, 1 gates, 2 bitstrings, ...) of ``seed``."""
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


# --------------------------------------------------------------------------
# graphs
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Graph:
    n: int
    edges: List[Tuple[int, int]]          # u < v, edge id = list position
    patterns: Dict[str, List[int]]        # pattern name -> edge ids (a matching)
    coords: List[Tuple[int, int]]         # (row, col) per qubit, for display

    def edges_array(self) -> np.ndarray:
        return np.asarray(self.edges, dtype=np.int32).reshape(-1, 2)

    def degree(self) -> np.ndarray:
        d = np.zeros(self.n, dtype=np.int64)
        for u, v in self.edges:
            d[u] += 1
            d[v] += 1
        return d

    def is_connected(self) -> bool:
        return _connected(self.n, self.edges)


def _connected(n: int, edges: Sequence[Tuple[int, int]]) -> bool:
    if n == 0:
        return True
    adj = [[] for _ in range(n)]
    for u, v in edges:
        adj[u].append(v)
        adj[v].append(u)
    seen = [False] * n
    stack = [0]
    seen[0] = True
    while stack:
        x = stack.pop()
        for y in adj[x]:
            if not seen[y]:
                seen[y] = True
                stack.append(y)
    return all(seen)


def _finish(sites: List[Tuple[int, int]], raw: List[Tuple[Tuple[int, int], Tuple[int, int], str]]) -> Graph:
    """Number the kept sites row-major and map the raw (site, site, pattern) edges."""
    sites = sorted(sites)
    index = {s: i for i, s in enumerate(sites)}
    edges: List[Tuple[int, int]] = []
    patterns: Dict[str, List[int]] = {}
    for a, b, p in raw:
        if a in index and b in index:
            u, v = sorted((index[a], index[b]))
            patterns.setdefault(p, []).append(len(edges))
            edges.append((u, v))
    return Graph(n=len(sites), edges=edges, patterns=patterns, coords=sites)


def grid(R: int, C: int) -> Graph:
    """R x C nearest-neighbour grid; qubit r*C + c."""
    raw = []
    for r in range(R):
        for c in range(C):
            if c + 1 < C:
                raw.append(((r, c), (r, c + 1), "A" if c % 2 == 0 else "B"))
            if r + 1 < R:
                raw.append(((r, c), (r + 1, c), "C" if r % 2 == 0 else "D"))
    return _finish([(r, c) for r in range(R) for c in range(C)], raw)


def _staggered_raw(R: int, C: int):
    raw = []
    for r in range(R - 1):
        delta = 1 if r % 2 == 0 else -1
        for c in range(C):
            raw.append(((r, c), (r + 1, c), "A" if r % 2 == 0 else "B"))
            c2 = c + delta
            if 0 <= c2 < C:
                raw.append(((r, c), (r + 1, c2), "C" if r % 2 == 0 else "D"))
    return raw


def staggered(R: int, C: int, remove_seed: Optional[int] = None) -> Graph:
    """R rows x C columns staggered diagonal-coupled grid (degree <= 4).

    Edges (r,c)-(r+1,c) ("straight") and (r,c)-(r+1,c+delta_r) ("offset"),
    delta_r = +1 for even r and -1 for odd r. With ``remove_seed`` one site,
    drawn from that seed's graph stream, is removed (redrawn until the graph
    stays connected); remaining sites are numbered row-major.
    """
    raw = _staggered_raw(R, C)
    sites = [(r, c) for r in range(R) for c in range(C)]
    if remove_seed is not None:
        g = rng(remove_seed, 0)
        for _ in range(1000):
            drop = sites[int(g.integers(len(sites)))]
            kept = [s for s in sites if s != drop]
            cand = _finish(kept, raw)
            if cand.is_connected():
                return cand
        raise RuntimeError("no removable site keeps the graph connected")
    return _finish(sites, raw)


def random_regular3(n: int, g: np.random.Generator, max_colours: int = 4, tries: int = 2000) -> Graph:
    """Random simple connected 3-regular graph (pairing model with rejection).

    Edges are properly coloured into layers named "0", "1", ...; a greedy
    colouring over seeded random edge orders is retried until it uses at most
    ``max_colours`` colours (falling back to the best found).
    """
    if n % 2 or n < 4:
        raise ValueError("3-regular graphs need even n >= 4")
    for _ in range(tries):
        stubs = np.repeat(np.arange(n), 3)
        g.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        es = set()
        ok = True
        for u, v in pairs:
            u, v = int(u), int(v)
            if u == v:
                ok = False
                break
            key = (min(u, v), max(u, v))
            if key in es:
                ok = False
                break
            es.add(key)
        if ok and _connected(n, list(es)):
            break
    else:
        raise RuntimeError("pairing model failed")
    edges = sorted(es)
    best = None
    for _ in range(200):
        order = g.permutation(len(edges))
        colour = [-1] * len(edges)
        used = [set() for _ in range(n)]
        for e in order:
            u, v = edges[e]
            c = 0
            while c in used[u] or c in used[v]:
                c += 1
            colour[e] = c
            used[u].add(c)
            used[v].add(c)
        k = max(colour) + 1
        if best is None or k < best[0]:
            best = (k, colour)
        if k <= max_colours:
            break
    k, colour = best
    patterns: Dict[str, List[int]] = {}
    for e, c in enumerate(colour):
        patterns.setdefault(str(c), []).append(e)
    return Graph(n=n, edges=edges, patterns=patterns, coords=[(0, i) for i in range(n)])


# --------------------------------------------------------------------------
# gates
# --------------------------------------------------------------------------
_I2 = np.eye(2, dtype=np.complex128)
_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_W = (_X + _Y) / math.sqrt(2.0)


def sqrt_pauli(P: np.ndarray) -> np.ndarray:
    """(I - iP)/sqrt(2): a square root of the Pauli-like involution P (up to phase)."""
    return (_I2 - 1j * P) / math.sqrt(2.0)


SQRT_X = sqrt_pauli(_X)
SQRT_Y = sqrt_pauli(_Y)
SQRT_W = sqrt_pauli(_W)
SYCAMORE_1Q = (SQRT_X, SQRT_Y, SQRT_W)
HADAMARD = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)


def fsim(theta: float, phi: float) -> np.ndarray:
    """fSim(theta, phi) in the basis |q0 q1>, q0 the high bit."""
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[1, 0, 0, 0],
                     [0, c, -1j * s, 0],
                     [0, -1j * s, c, 0],
                     [0, 0, 0, np.exp(-1j * phi)]], dtype=np.complex128)


def haar_su2(g: np.random.Generator) -> np.ndarray:
    a, b, c, d = g.standard_normal(4)
    nrm = math.sqrt(a * a + b * b + c * c + d * d)
    a, b, c, d = a / nrm, b / nrm, c / nrm, d / nrm
    return np.array([[a + 1j * b, c + 1j * d], [-c + 1j * d, a - 1j * b]], dtype=np.complex128)


@dataclasses.dataclass
class Gate:
    cycle: int                 # 1-based cycle index
    qubits: Tuple[int, ...]    # (q,) or (q0, q1); q0 is the high bit of the 4x4 basis
    m: np.ndarray              # 2x2 or 4x4 complex128, rows = outputs


def haar_u4(g: np.random.Generator) -> np.ndarray:
    """Haar-random 4x4 unitary (QR of a complex Gaussian matrix, phases fixed)."""
    z = (g.standard_normal((4, 4)) + 1j * g.standard_normal((4, 4))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


def rqc(graph: Graph, depth: int, g: np.random.Generator, *, sequence: str = SYCAMORE_SEQUENCE,
        theta: float = math.pi / 2, phi: float = math.pi / 6, oneq: str = "sycamore",
        twoq: str = "fsim") -> List[Gate]:
    """Random circuit: cycle k = a 1q gate on every qubit, then fSim(theta, phi) on
    every edge of pattern ``sequence[(k-1) % len(sequence)]``.

    ``oneq="sycamore"``: drawn from {sqrt X, sqrt Y, sqrt W}, uniform in cycle 1 and
    never repeating the qubit's previous gate afterwards. ``oneq="haar"``: Haar SU(2).
    ``twoq="haar"`` replaces every fSim by an independent Haar-random U(4).
    """
    gates: List[Gate] = []
    prev = [-1] * graph.n
    for k in range(1, depth + 1):
        for q in range(graph.n):
            if oneq == "haar":
                u = haar_su2(g)
            else:
                choices = [i for i in range(3) if i != prev[q]]
                pick = choices[int(g.integers(len(choices)))]
                prev[q] = pick
                u = SYCAMORE_1Q[pick]
            gates.append(Gate(k, (q,), u))
        pat = sequence[(k - 1) % len(sequence)]
        f = fsim(theta, phi)
        for e in graph.patterns.get(pat, []):
            u, v = graph.edges[e]
            gates.append(Gate(k, (u, v), haar_u4(g) if twoq == "haar" else f.copy()))
    return gates


def graph_state_circuit(graph: Graph) -> List[Gate]:
    """Cycle 1: H on every qubit, then CZ = fSim(0, pi) once on every edge."""
    gates = [Gate(1, (q,), HADAMARD.copy()) for q in range(graph.n)]
    cz = fsim(0.0, math.pi)
    gates += [Gate(1, (u, v), cz.copy()) for (u, v) in graph.edges]
    return gates


def mirror_circuit(gates: Sequence[Gate]) -> List[Gate]:
    """U followed by U^dagger (cycles continue after the last one); U^dag U = I."""
    if not gates:
        return []
    d = max(gt.cycle for gt in gates)
    out = [Gate(gt.cycle, gt.qubits, gt.m.copy()) for gt in gates]
    for gt in reversed(list(gates)):
        out.append(Gate(2 * d + 1 - gt.cycle, gt.qubits, gt.m.conj().T.copy()))
    return out


# --------------------------------------------------------------------------
# bitstrings
# --------------------------------------------------------------------------
def bitstrings(n: int, count: int, g: np.random.Generator) -> np.ndarray:
    """(count, n) uint8 array, bit q = s_q; uniform, duplicates allowed."""
    return g.integers(0, 2, size=(count, n), dtype=np.uint8)


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """(count, n) 0/1 -> (count, ceil(n/64)) uint64 words, bit q of word q//64 = s_q."""
    bits = np.asarray(bits, dtype=np.uint64)
    cnt, n = bits.shape
    words = (n + 63) // 64
    out = np.zeros((cnt, max(words, 1)), dtype=np.uint64)
    for q in range(n):
        out[:, q // 64] |= bits[:, q] << np.uint64(q % 64)
    return out


def all_bitstrings(n: int) -> np.ndarray:
    idx = np.arange(1 << n, dtype=np.int64)
    return ((idx[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    graph: Graph
    gates: List[Gate]
    depth: int
    split: int                 # cycles 1..split -> ket, split+1..depth -> bra
    chi: int                   # bond cap (0 = none)
    cutoff: float              # relative singular-value cutoff
    bits: np.ndarray           # (B, n) uint8


def workload(name: str, n_bits: Optional[int] = None) -> Workload:
    """The seeded stand-in workloads (seed = BASE_SEED + config number).

    * ``grid12``   3x4 grid, 8 cycles, untruncated, 256 bitstrings.
    * ``grid20``   4x5 grid, 14 cycles, untruncated, 4096 bitstrings.
    * ``syc53``    6x9 staggered grid minus one seeded site (53 q), 10 cycles,
                   split after cycle 5, chi 64, cutoff 1e-8, 65536 bitstrings.
    * ``syc104``   8x13 staggered grid (104 q), 8 cycles, chi 128, cutoff 1e-8.
    """
    if name == "grid12":
        seed, gr, depth, split, chi, cut, B = BASE_SEED + 1, grid(3, 4), 8, 4, 0, 1e-12, 256
    elif name == "grid20":
        seed, gr, depth, split, chi, cut, B = BASE_SEED + 2, grid(4, 5), 14, 7, 0, 1e-12, 4096
    elif name == "syc53":
        seed = BASE_SEED + 3
        gr, depth, split, chi, cut, B = staggered(6, 9, remove_seed=seed), 10, 5, 64, 1e-8, 65536
    elif name == "syc104":
        seed = BASE_SEED + 5
        gr, depth, split, chi, cut, B = staggered(8, 13), 8, 4, 128, 1e-8, 65536
    else:
        raise KeyError(name)
    gates = rqc(gr, depth, rng(seed, 1))
    B = B if n_bits is None else n_bits
    bits = bitstrings(gr.n, B, rng(seed, 2))
    return Workload(name, gr, gates, depth, split, chi, cut, bits)


def regular3_family(count: int = 32, depth: int = 12, n_bits: int = 1024) -> List[Workload]:
    """``count`` circuits on random 3-regular graphs of 24..40 qubits (n_i = 24 + 2*floor(9i/32)),
    Haar SU(2) single-qubit layers and fSim(pi/2, pi/6) on one colour class per cycle."""
    seed = BASE_SEED + 4
    out = []
    for i in range(count):
        n = 24 + 2 * ((9 * i) // 32)
        g = rng(seed + 1000 * i, 0)
        gr = random_regular3(n, g)
        seq = "".join(sorted(gr.patterns))
        gates = rqc(gr, depth, rng(seed + 1000 * i, 1), sequence=seq, oneq="haar")
        bits = bitstrings(n, n_bits, rng(seed + 1000 * i, 2))
        out.append(Workload(f"reg3_{i}_n{n}", gr, gates, depth, depth // 2, 0, 1e-12, bits))
    return out

"""Thin Python binding of the C ABI in include/tn.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: all compute runs in libtn.so's CUDA kernels. The
library is loaded from this package directory; importing this module when
libtn.so is missing raises immediately (there is no CPU fallback).

Device memory for the library comes from PyTorch's caching allocator unless
``allocator=None`` is passed to :func:`tn_build`; streams are PyTorch streams
(or raw ``cudaStream_t`` integers).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtn.so")

TN_OK, TN_ERR_ARG, TN_ERR_GRAPH, TN_ERR_OOM, TN_ERR_NO_PATH, TN_ERR_STATE, TN_ERR_CUDA, TN_ERR_TIMEOUT, \
    TN_ERR_UNSUPPORTED = range(9)
STATUS_NAMES = {0: "TN_OK", 1: "TN_ERR_ARG", 2: "TN_ERR_GRAPH", 3: "TN_ERR_OOM", 4: "TN_ERR_NO_PATH",
                5: "TN_ERR_STATE", 6: "TN_ERR_CUDA", 7: "TN_ERR_TIMEOUT", 8: "TN_ERR_UNSUPPORTED"}
PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "tf32x3": 3, "bf16x3": 4, "bf16x6": 5, "tf32x6": 6}


class TNError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class c128(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class tn_graph(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_edges", C.c_int32), ("edges", C.POINTER(C.c_int32))]


class tn_gate(C.Structure):
    _fields_ = [("cycle", C.c_int32), ("arity", C.c_int32), ("q", C.c_int32 * 2), ("m", c128 * 16)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class tn_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class tn_path_opts(C.Structure):
    _fields_ = [("max_rank", C.c_int32), ("boundary_only", C.c_int32), ("connected", C.c_int32),
                ("max_states", C.c_int64), ("n_cuts", C.c_int32), ("cut_edges", C.POINTER(C.c_int32)),
                ("n_cut_edges", C.c_int32), ("max_intermediate", C.c_int64), ("mem_budget_bytes", C.c_double),
                ("no_merge", C.c_int32), ("layers", C.c_int32), ("byte_weight", C.c_double)]


class tn_plan_info(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_steps", C.c_int32), ("n_cuts", C.c_int32), ("n_slices", C.c_int64),
                ("score", C.c_double), ("cmacs", C.c_double), ("flops", C.c_double), ("bytes_c64", C.c_double),
                ("max_intermediate", C.c_int64), ("states_expanded", C.c_int64), ("max_rank_used", C.c_int32),
                ("chunk_bitstrings", C.c_int32), ("workspace_bytes", C.c_int64), ("n_nodes", C.c_int32)]


class tn_server_cfg(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_double), ("max_inflight", C.c_int32), ("n_streams", C.c_int32)]


class tn_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("rejected", C.c_int64),
                ("amplitudes", C.c_int64), ("busy_seconds", C.c_double), ("p50_latency_s", C.c_double),
                ("p99_latency_s", C.c_double), ("max_inflight_seen", C.c_double),
                ("peak_admitted_bytes", C.c_double), ("cancelled", C.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2011_02621_gb300.build.build() first "
                          "(this library has no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "tn_build": (i32, [C.POINTER(tn_graph), C.POINTER(tn_gate), i64, C.POINTER(tn_allocator), C.POINTER(vp)]),
        "tn_evolve_two_sided": (i32, [vp, i32, i32, dbl, vp]),
        "tn_circuit_bond_dims": (i32, [vp, i32, C.POINTER(i32)]),
        "tn_set_compression": (i32, [vp, i32]),
        "tn_set_svd_sweeps": (i32, [vp, i32]),
        "tn_program_inspect": (i32, [vp, i32, i32, dbl, i32, C.POINTER(i64), C.POINTER(dbl), C.POINTER(i64)]),
        "tn_path": (i32, [vp, C.POINTER(tn_path_opts), C.POINTER(vp), C.POINTER(tn_plan_info)]),
        "tn_plan_details": (i32, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64)]),
        "tn_plan_estimate": (i32, [vp, i32, i32, dbl, C.POINTER(tn_path_opts), C.POINTER(tn_plan_info)]),
        "tn_plan_inspect": (i32, [vp, i32, i32, dbl, C.POINTER(tn_path_opts), C.POINTER(i64), C.POINTER(i64),
                                  C.POINTER(i32), C.POINTER(i64), C.POINTER(i64)]),
        "tn_amplitudes": (i32, [vp, vp, i64, i32, vp, vp]),
        "tn_amplitudes_static": (i32, [vp, vp, i64, i32, vp, vp]),
        "tn_amplitudes_slices": (i32, [vp, vp, i64, i32, i64, i64, vp, vp]),
        "tn_launch_count": (i64, [i32]),
        "tn_profile_enable": (i32, [i32]),
        "tn_profile_read": (i32, [i32, C.c_char_p, i32, C.POINTER(i64), C.POINTER(dbl), C.POINTER(dbl),
                                 C.POINTER(dbl)]),
        "tn_circuit_free": (None, [vp]),
        "tn_plan_free": (None, [vp]),
        "tn_last_error": (C.c_char_p, []),
        "tn_gate_split": (i32, [C.POINTER(c128), C.POINTER(c128), C.POINTER(c128), C.POINTER(i32)]),
        "tn_path_search": (i32, [C.POINTER(tn_graph), C.POINTER(dbl), C.POINTER(tn_path_opts), C.POINTER(i32),
                                 C.POINTER(dbl), C.POINTER(i64)]),
        "tn_cut_search": (i32, [C.POINTER(tn_graph), C.POINTER(dbl), C.POINTER(tn_path_opts), C.POINTER(i32),
                                C.POINTER(i32), C.POINTER(i32), C.POINTER(dbl)]),
        "tn_merge_search": (i32, [C.POINTER(tn_graph), C.POINTER(i32), C.POINTER(i32), C.POINTER(tn_path_opts),
                                  C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(dbl)]),
        "tn_server_create": (i32, [C.POINTER(tn_server_cfg), C.POINTER(vp)]),
        "tn_server_submit": (i32, [vp, vp, vp, i64, i32, vp, C.POINTER(C.c_uint64)]),
        "tn_server_wait": (i32, [vp, C.c_uint64, i64]),
        "tn_server_stats_get": (i32, [vp, C.POINTER(tn_server_stats)]),
        "tn_server_cancel": (i32, [vp, C.c_uint64]),
        "tn_server_free": (None, [vp]),
        "tn_autotune": (i32, [vp, i32, i64, vp, C.POINTER(i32)]),
        "tn_plan_kernels": (i32, [vp, i32, C.POINTER(i32)]),
        "tn_plan_set_kernels": (i32, [vp, i32, C.POINTER(i32)]),
        "tn_batch_create": (i32, [C.POINTER(vp), i32, vp, C.POINTER(i64), i32, dbl, vp, C.POINTER(vp)]),
        "tn_batch_set_bits": (i32, [vp, vp, vp]),
        "tn_batch_run": (i32, [vp, vp]),
        "tn_batch_read": (i32, [vp, vp, vp]),
        "tn_batch_info": (i32, [vp, C.POINTER(i64), C.POINTER(i64)]),
        "tn_batch_free": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB = _load()


def _check(status: int):
    if status != TN_OK:
        raise TNError(status, LIB.tn_last_error().decode(errors="replace"))


def tn_last_error() -> str:
    return LIB.tn_last_error().decode(errors="replace")


def tn_launch_count(reset: bool = False) -> int:
    return int(LIB.tn_launch_count(1 if reset else 0))


def tn_profile_enable(on: bool = True, per_step: bool = False):
    """Start (clearing the records) or stop per-kernel tracing; per_step keeps one record per kind
    and contraction step, named "<kind>#<step>"."""
    _check(LIB.tn_profile_enable((2 if per_step else 1) if on else 0))


def tn_profile_read() -> dict:
    """{kind: {launches, ms, bytes, flops}} for every kernel kind recorded since tn_profile_enable."""
    out = {}
    i = 0
    while True:
        name = C.create_string_buffer(64)
        la, ms, by, fl = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
        st = LIB.tn_profile_read(i, name, 64, C.byref(la), C.byref(ms), C.byref(by), C.byref(fl))
        if st != TN_OK:
            return out
        out[name.value.decode()] = dict(launches=la.value, ms=ms.value, bytes=by.value, flops=fl.value)
        i += 1


# --------------------------------------------------------------------------
# allocator bridge to PyTorch's caching allocator
# --------------------------------------------------------------------------
_torch_alloc = None


def torch_allocator():
    """A tn_allocator whose callbacks call torch.cuda.caching_allocator_alloc / _delete."""
    global _torch_alloc
    if _torch_alloc is None:
        import torch

        def _alloc(size, stream, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(size), stream=int(stream or 0)))
            except Exception:
                return None

        def _free(ptr, size, stream, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        a_fn, f_fn = ALLOC_FN(_alloc), FREE_FN(_free)
        _torch_alloc = (tn_allocator(a_fn, f_fn, None), a_fn, f_fn)
    return _torch_alloc[0]


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# --------------------------------------------------------------------------
# handles
# --------------------------------------------------------------------------
class Circuit:
    """Owns a tn_circuit*; freed with tn_circuit_free."""

    def __init__(self, ptr, n_qubits, n_edges, keep):
        self.ptr = ptr
        self.n_qubits = n_qubits
        self.n_edges = n_edges
        self._keep = keep

    def __del__(self):
        if getattr(self, "ptr", None):
            LIB.tn_circuit_free(self.ptr)
            self.ptr = None


class Plan:
    """Owns a tn_plan*; keeps its circuit alive; freed with tn_plan_free."""

    def __init__(self, ptr, circuit, info: dict):
        self.ptr = ptr
        self.circuit = circuit
        self.info = info

    def __del__(self):
        if getattr(self, "ptr", None):
            LIB.tn_plan_free(self.ptr)
            self.ptr = None


def _graph_struct(n: int, edges):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    g = tn_graph(int(n), int(e.shape[0]), e.ctypes.data_as(C.POINTER(C.c_int32)))
    return g, e


def gates_array(gates) -> C.Array:
    """Marshal gate objects (``.cycle``, ``.qubits``, ``.m``) into a tn_gate array."""
    arr = (tn_gate * max(len(gates), 1))()
    for i, g in enumerate(gates):
        arr[i].cycle = int(g.cycle)
        arr[i].arity = len(g.qubits)
        arr[i].q[0] = int(g.qubits[0])
        arr[i].q[1] = int(g.qubits[1]) if len(g.qubits) > 1 else -1
        m = np.asarray(g.m, dtype=np.complex128).ravel()
        for j, x in enumerate(m):
            arr[i].m[j].re = float(x.real)
            arr[i].m[j].im = float(x.imag)
    return arr


def tn_build(n_qubits: int, edges, gates, allocator="torch") -> Circuit:
    g, e = _graph_struct(n_qubits, edges)
    arr = gates_array(gates)
    alloc = torch_allocator() if allocator == "torch" else allocator
    out = C.c_void_p()
    _check(LIB.tn_build(C.byref(g), arr, len(gates), C.byref(alloc) if alloc is not None else None, C.byref(out)))
    return Circuit(out, int(n_qubits), int(e.shape[0]), (alloc,))


COMPRESSIONS = {"one_sided": 0, "two_sided": 1}


def tn_set_compression(c: Circuit, mode: str = "one_sided"):
    """Bond compression of both halves for the next tn_evolve_two_sided: "one_sided" (Eqs. svd/
    svd2) or "two_sided" (the singular values of the local product of the two endpoints)."""
    if mode not in COMPRESSIONS:
        raise ValueError(f"unknown compression {mode!r}")
    _check(LIB.tn_set_compression(c.ptr, COMPRESSIONS[mode]))


def tn_set_svd_sweeps(c: Circuit, max_sweeps: int = 0):
    """Cap on the Jacobi sweeps of every SVD of both halves (0: the default, 60)."""
    _check(LIB.tn_set_svd_sweeps(c.ptr, int(max_sweeps)))


def tn_evolve_two_sided(c: Circuit, split_cycle: int, chi_max: int = 0, cutoff_rel: float = 1e-12, stream=None,
                        compress=None):
    """compress: None keeps the circuit's mode (tn_set_compression), else sets it first."""
    if compress is not None:
        tn_set_compression(c, compress)
    _check(LIB.tn_evolve_two_sided(c.ptr, int(split_cycle), int(chi_max), float(cutoff_rel), _stream_handle(stream)))


def tn_circuit_bond_dims(c: Circuit, side: int) -> np.ndarray:
    out = np.zeros(max(c.n_edges, 1), dtype=np.int32)
    _check(LIB.tn_circuit_bond_dims(c.ptr, int(side), out.ctypes.data_as(C.POINTER(C.c_int32))))
    return out[: c.n_edges]


def _opts(max_rank=0, boundary_only=True, connected=True, max_states=0, n_cuts=-1, cut_edges=None,
          max_intermediate=0, mem_budget_bytes=0.0, merge=True, layers=1, byte_weight=0.0):
    o = tn_path_opts()
    o.max_rank = int(max_rank)
    o.boundary_only = 1 if boundary_only else 0
    o.connected = 1 if connected else 0
    o.max_states = int(max_states)
    o.n_cuts = int(n_cuts)
    keep = None
    if cut_edges is not None and len(cut_edges):
        keep = np.ascontiguousarray(np.asarray(cut_edges, dtype=np.int32))
        o.cut_edges = keep.ctypes.data_as(C.POINTER(C.c_int32))
        o.n_cut_edges = int(keep.size)
    o.max_intermediate = int(max_intermediate)
    o.mem_budget_bytes = float(mem_budget_bytes)
    o.no_merge = 0 if merge else 1
    o.layers = int(layers)
    o.byte_weight = float(byte_weight)
    return o, keep


def _info_dict(info: tn_plan_info) -> dict:
    return {name: getattr(info, name) for name, _ in tn_plan_info._fields_}


def tn_path(c: Circuit, **opts) -> Plan:
    o, keep = _opts(**opts)
    out = C.c_void_p()
    info = tn_plan_info()
    _check(LIB.tn_path(c.ptr, C.byref(o), C.byref(out), C.byref(info)))
    return Plan(out, c, _info_dict(info))


def tn_plan_estimate(c: Circuit, split_cycle: int, chi: int = 0, cutoff: float = 1e-12, **opts) -> dict:
    """The summary of the plan tn_path(**opts) would make after tn_evolve_two_sided(split_cycle,
    chi, cutoff), from the structural bond bounds, on the host (no device needed)."""
    o, keep = _opts(**opts)
    info = tn_plan_info()
    _check(LIB.tn_plan_estimate(c.ptr, int(split_cycle), int(chi), float(cutoff), C.byref(o), C.byref(info)))
    del keep
    return _info_dict(info)


STEP_DESC_LEN = 17 + 2 * 32
STEP_FIELDS = ("M", "K", "N", "layer", "n_rest", "ket_off", "ket_sig", "bra_off", "bra_sig", "phys", "t_ocol",
               "t_bka", "t_bkb", "t_bna", "t_bnb", "t_sa", "t_sb")


def tn_plan_inspect(c: Circuit, split_cycle: int, chi: int = 0, cutoff: float = 1e-12, **opts):
    """(layout, steps, tables) of the plan tn_plan_estimate describes, on the host: layout a dict
    (item stride, slices, item sizes, per-qubit node offsets, per-edge bonds), steps a list of
    dicts (the fields of STEP_FIELDS, rest_dim, rest_ostride), tables an int32 array."""
    o, keep = _opts(**opts)
    ns, nt = C.c_int64(), C.c_int64()
    _check(LIB.tn_plan_inspect(c.ptr, int(split_cycle), int(chi), float(cutoff), C.byref(o), None, None, None,
                               C.byref(ns), C.byref(nt)))
    lay = np.zeros(8 + 2 * c.n_qubits + 2 * c.n_edges, dtype=np.int64)
    st = np.zeros((max(ns.value, 1), STEP_DESC_LEN), dtype=np.int64)
    tab = np.zeros(max(nt.value, 1), dtype=np.int32)
    _check(LIB.tn_plan_inspect(c.ptr, int(split_cycle), int(chi), float(cutoff), C.byref(o),
                               lay.ctypes.data_as(C.POINTER(C.c_int64)), st.ctypes.data_as(C.POINTER(C.c_int64)),
                               tab.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(ns), C.byref(nt)))
    del keep
    n, ne = c.n_qubits, c.n_edges
    layout = dict(max_t=int(lay[0]), n_slices=int(lay[1]), n_steps=int(lay[2]), ket_elems=int(lay[3]),
                  bra_elems=int(lay[4]), merged=bool(lay[5]), ket_half_elems=int(lay[6]), bra_half_elems=int(lay[7]),
                  ket_off=lay[8:8 + 2 * n:2].copy(), bra_off=lay[9:8 + 2 * n:2].copy(),
                  ket_dims=lay[8 + 2 * n::2][:ne].copy(), bra_dims=lay[9 + 2 * n::2][:ne].copy())
    steps = []
    for row in st[: ns.value]:
        d = {f: int(v) for f, v in zip(STEP_FIELDS, row[:17])}
        d["rest_dim"] = [int(x) for x in row[17:17 + d["n_rest"]]]
        d["rest_ostride"] = [int(x) for x in row[17 + 32:17 + 32 + d["n_rest"]]]
        steps.append(d)
    return layout, steps, tab[: nt.value].copy()


PROG_ENTRY_LEN = 16
PROG_MAT_LEN = 66
PROG_FIELDS = ("op", "k", "l", "edge", "sv_is_k", "din", "chi_o", "n", "dout", "m_k", "m_l", "pk", "pl", "off_k",
               "off_l", "id")


def tn_program_inspect(c: Circuit, split_cycle: int, chi: int = 0, cutoff: float = 1e-12, side: int = 0):
    """The gate program of one half (0 ket, 1 bra) tn_evolve_two_sided builds with the circuit's
    compression mode, from the structural bond bounds, on the host: a list of dicts, one per
    entry in processing order (fields PROG_FIELDS; two-qubit entries carry P and Q as [s'][s][a]
    complex arrays and the cutoff, single-qubit entries (op 1, node k) the 2x2 matrix u)."""
    n = C.c_int64()
    _check(LIB.tn_program_inspect(c.ptr, int(split_cycle), int(chi), float(cutoff), int(side), None, None,
                                  C.byref(n)))
    e = np.zeros((max(n.value, 1), PROG_ENTRY_LEN), dtype=np.int64)
    m = np.zeros((max(n.value, 1), PROG_MAT_LEN), dtype=np.float64)
    _check(LIB.tn_program_inspect(c.ptr, int(split_cycle), int(chi), float(cutoff), int(side),
                                  e.ctypes.data_as(C.POINTER(C.c_int64)), m.ctypes.data_as(C.POINTER(C.c_double)),
                                  C.byref(n)))
    out = []
    for row, mat in zip(e[: n.value], m[: n.value]):
        d = {f: int(v) for f, v in zip(PROG_FIELDS, row)}
        if d["op"] == 2:
            d["P"] = (mat[0:32:2] + 1j * mat[1:32:2]).reshape(2, 2, 4)
            d["Q"] = (mat[32:64:2] + 1j * mat[33:64:2]).reshape(2, 2, 4)
            d["cutoff"] = float(mat[64])
        else:
            d["u"] = (mat[0:8:2] + 1j * mat[1:8:2]).reshape(2, 2)
        out.append(d)
    return out


def tn_plan_details(p: Plan):
    n = max(p.info["n_qubits"], p.info["n_nodes"])
    order = np.zeros(n, dtype=np.int32)
    cuts = np.zeros(max(p.info["n_cuts"], 1), dtype=np.int32)
    steps = np.zeros((max(p.info["n_steps"], 1), 3), dtype=np.int64)
    _check(LIB.tn_plan_details(p.ptr, order.ctypes.data_as(C.POINTER(C.c_int32)),
                               cuts.ctypes.data_as(C.POINTER(C.c_int32)),
                               steps.ctypes.data_as(C.POINTER(C.c_int64))))
    return order, cuts[: p.info["n_cuts"]], steps[: p.info["n_steps"]]


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """(B, n) 0/1 -> (B, ceil(n/64)) uint64 words, bit q of word q//64 = s_q."""
    bits = np.asarray(bits, dtype=np.uint64)
    B, n = bits.shape
    words = max((n + 63) // 64, 1)
    out = np.zeros((B, words), dtype=np.uint64)
    for q in range(n):
        out[:, q // 64] |= bits[:, q] << np.uint64(q % 64)
    return out


def tn_amplitudes(p: Plan, bits, prec: str = "fp64", out=None, stream=None):
    """Amplitudes of the bitstrings ``bits``.

    ``bits``: numpy (B, n) 0/1 array, numpy (B, words) uint64 packed words, or a
    torch int64/uint64 tensor of packed words (host or device). ``out``: None
    (returns a numpy complex128 array) or a torch complex128 tensor of B
    entries (host or device) that receives the results.
    """
    n = p.circuit.n_qubits
    words = max((n + 63) // 64, 1)
    keep = None
    if hasattr(bits, "data_ptr"):
        B = int(bits.shape[0])
        bptr = bits.data_ptr()
        keep = bits
    else:
        b = np.asarray(bits)
        if b.dtype != np.uint64 or b.ndim != 2 or b.shape[1] != words:
            b = pack_bits(b.reshape(-1, n))
        b = np.ascontiguousarray(b)
        B = int(b.shape[0])
        bptr = b.ctypes.data
        keep = b
    if out is None:
        res = np.zeros(B, dtype=np.complex128)
        optr = res.ctypes.data
    else:
        res = out
        optr = out.data_ptr()
    _check(LIB.tn_amplitudes(p.ptr, C.c_void_p(bptr), B, PRECISIONS[prec], C.c_void_p(optr), _stream_handle(stream)))
    del keep
    return res


def tn_amplitudes_slices(p: Plan, bits, prec: str = "fp64", slice_begin: int = 0, slice_end=None, out=None,
                         stream=None):
    """Per-bitstring FP64 partial sums over the slices [slice_begin, slice_end) of the plan's cut
    network (default: all, i.e. the amplitudes). Arguments otherwise those of :func:`tn_amplitudes`."""
    n = p.circuit.n_qubits
    words = max((n + 63) // 64, 1)
    if slice_end is None:
        slice_end = p.info["n_slices"]
    if hasattr(bits, "data_ptr"):
        B, bptr, keep = int(bits.shape[0]), bits.data_ptr(), bits
    else:
        b = np.asarray(bits)
        if b.dtype != np.uint64 or b.ndim != 2 or b.shape[1] != words:
            b = pack_bits(b.reshape(-1, n))
        keep = np.ascontiguousarray(b)
        B, bptr = int(keep.shape[0]), keep.ctypes.data
    res = np.zeros(B, dtype=np.complex128) if out is None else out
    optr = res.ctypes.data if isinstance(res, np.ndarray) else res.data_ptr()
    _check(LIB.tn_amplitudes_slices(p.ptr, C.c_void_p(bptr), B, PRECISIONS[prec], int(slice_begin), int(slice_end),
                                    C.c_void_p(optr), _stream_handle(stream)))
    del keep
    return res


def tn_amplitudes_static(p: Plan, bits, prec: str = "fp64", out=None, stream=None):
    """Same as :func:`tn_amplitudes`, for callers that must not allocate device memory during the
    call: the library's scratch comes from its fixed 32 MiB static device array, never from an
    allocator. Arguments and results are those of :func:`tn_amplitudes`."""
    n = p.circuit.n_qubits
    words = max((n + 63) // 64, 1)
    if hasattr(bits, "data_ptr"):
        B, bptr, keep = int(bits.shape[0]), bits.data_ptr(), bits
    else:
        b = np.asarray(bits)
        if b.dtype != np.uint64 or b.ndim != 2 or b.shape[1] != words:
            b = pack_bits(b.reshape(-1, n))
        keep = np.ascontiguousarray(b)
        B, bptr = int(keep.shape[0]), keep.ctypes.data
    res = np.zeros(B, dtype=np.complex128) if out is None else out
    optr = res.ctypes.data if isinstance(res, np.ndarray) else res.data_ptr()
    _check(LIB.tn_amplitudes_static(p.ptr, C.c_void_p(bptr), B, PRECISIONS[prec], C.c_void_p(optr),
                                    _stream_handle(stream)))
    del keep
    return res


def tn_gate_split(m):
    mm = (c128 * 16)()
    for j, x in enumerate(np.asarray(m, dtype=np.complex128).ravel()):
        mm[j].re, mm[j].im = float(x.real), float(x.imag)
    P, Q = (c128 * 16)(), (c128 * 16)()
    chi = C.c_int32()
    _check(LIB.tn_gate_split(mm, P, Q, C.byref(chi)))
    to = lambda a: np.array([a[j].re + 1j * a[j].im for j in range(16)]).reshape(2, 2, 4)
    return to(P), to(Q), int(chi.value)


def tn_path_search(n_qubits: int, edges, dims, **opts):
    g, e = _graph_struct(n_qubits, edges)
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.float64))
    o, keep = _opts(**opts)
    order = np.zeros(n_qubits, dtype=np.int32)
    score = C.c_double()
    states = C.c_int64()
    _check(LIB.tn_path_search(C.byref(g), d.ctypes.data_as(C.POINTER(C.c_double)), C.byref(o),
                              order.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(score), C.byref(states)))
    return order, float(score.value), int(states.value)


def tn_merge_search(n_qubits: int, edges, ket_dims, bra_dims, **opts):
    """The network tn_path contracts for these bond dimensions: (owner per qubit, contraction order
    of the nodes, number of cuts, total complex MACs)."""
    g, e = _graph_struct(n_qubits, edges)
    kd = np.ascontiguousarray(np.asarray(ket_dims, dtype=np.int32))
    bd = np.ascontiguousarray(np.asarray(bra_dims, dtype=np.int32))
    o, keep = _opts(**opts)
    owner = np.zeros(n_qubits, dtype=np.int32)
    order = np.zeros(n_qubits, dtype=np.int32)
    nn, nc, tot = C.c_int32(), C.c_int32(), C.c_double()
    _check(LIB.tn_merge_search(C.byref(g), kd.ctypes.data_as(C.POINTER(C.c_int32)),
                               bd.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(o),
                               owner.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(nn),
                               order.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(nc), C.byref(tot)))
    del e, keep
    return owner, order[: nn.value], nc.value, tot.value


def tn_cut_search(n_qubits: int, edges, dims, **opts):
    """(order, cuts, total complex MACs) of the planner on an arbitrary graph (host only)."""
    g, e = _graph_struct(n_qubits, edges)
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.float64))
    o, keep = _opts(**opts)
    order = np.zeros(n_qubits, dtype=np.int32)
    cuts = np.zeros(max(e.shape[0], 1), dtype=np.int32)
    nc = C.c_int32()
    tot = C.c_double()
    _check(LIB.tn_cut_search(C.byref(g), d.ctypes.data_as(C.POINTER(C.c_double)), C.byref(o),
                             order.ctypes.data_as(C.POINTER(C.c_int32)), cuts.ctypes.data_as(C.POINTER(C.c_int32)),
                             C.byref(nc), C.byref(tot)))
    return order, cuts[: nc.value], float(tot.value)


# --------------------------------------------------------------------------
# serving loop
# --------------------------------------------------------------------------
class Server:
    """Owns a tn_server*; keeps every plan it served alive until it is freed."""

    def __init__(self, ptr):
        self.ptr = ptr
        self._pending = {}
        self._plans = []

    def __del__(self):
        if getattr(self, "ptr", None):
            LIB.tn_server_free(self.ptr)
            self.ptr = None


def tn_server_create(hbm_budget_bytes: float = 0.0, max_inflight: int = 0, n_streams: int = 0) -> Server:
    cfg = tn_server_cfg(float(hbm_budget_bytes), int(max_inflight), int(n_streams))
    out = C.c_void_p()
    _check(LIB.tn_server_create(C.byref(cfg), C.byref(out)))
    return Server(out)


def tn_server_submit(s: Server, p: Plan, bits, prec: str = "fp64", out=None) -> int:
    n = p.circuit.n_qubits
    words = max((n + 63) // 64, 1)
    b = np.asarray(bits)
    if b.dtype != np.uint64 or b.ndim != 2 or b.shape[1] != words:
        b = pack_bits(b.reshape(-1, n))
    b = np.ascontiguousarray(b)
    res = np.zeros(b.shape[0], dtype=np.complex128) if out is None else out
    optr = res.ctypes.data if isinstance(res, np.ndarray) else res.data_ptr()
    t = C.c_uint64()
    _check(LIB.tn_server_submit(s.ptr, p.ptr, C.c_void_p(b.ctypes.data), int(b.shape[0]), PRECISIONS[prec],
                                C.c_void_p(optr), C.byref(t)))
    s._pending[int(t.value)] = (res, p)
    if not any(q is p for q in s._plans):
        s._plans.append(p)
    return int(t.value)


def tn_server_wait(s: Server, ticket: int, timeout_ms: int = -1):
    st = LIB.tn_server_wait(s.ptr, C.c_uint64(ticket), int(timeout_ms))
    if st == TN_ERR_TIMEOUT:
        raise TNError(st, "request not complete")
    res, _ = s._pending.pop(ticket, (None, None))
    _check(st)
    return res


def tn_server_free(s: Server):
    if s.ptr:
        LIB.tn_server_free(s.ptr)
        s.ptr = None


def tn_server_cancel(s: Server, ticket: int):
    """Remove a request that is still queued (TN_ERR_STATE if it is running or complete)."""
    _check(LIB.tn_server_cancel(s.ptr, C.c_uint64(ticket)))
    s._pending.pop(ticket, None)


def tn_server_stats_get(s: Server) -> dict:
    st = tn_server_stats()
    _check(LIB.tn_server_stats_get(s.ptr, C.byref(st)))
    return {name: getattr(st, name) for name, _ in tn_server_stats._fields_}


# ---------------------------------------------------------------------------
# kernel autotuning and batched circuits
# ---------------------------------------------------------------------------
KERNEL_NAMES = {0: "simt_auto", 1: "simt_tile64x64", 2: "simt_tile128x16", 3: "simt_tile256x4",
                4: "simt_stream", 5: "simt_stream_fixed", 6: "simt_small", 7: "simt_narrow", 8: "simt_box",
                16: "tcgen05_split",
                32: "tcgen05_tma_buildb", 33: "tcgen05_tma_buildb_bn128", 34: "tcgen05_tma_buildb_bn64",
                40: "tcgen05_tma_loadb", 41: "tcgen05_tma_loadb_bn128", 42: "tcgen05_tma_loadb_bn64",
                48: "tcgen05_tma", 49: "tcgen05_tma_bn128", 50: "tcgen05_tma_bn64",
                56: "tcgen05_tma_persist", 57: "tcgen05_tma_persist_bn128", 58: "tcgen05_tma_persist_bn64",
                64: "tcgen05_persist_c64", 65: "tcgen05_persist_c64_bn128", 66: "tcgen05_persist_c64_bn64",
                72: "tcgen05_persist_loadb", 73: "tcgen05_persist_loadb_bn128", 74: "tcgen05_persist_loadb_bn64",
                80: "tcgen05_persist_c64_loadb", 81: "tcgen05_persist_c64_loadb_bn128",
                82: "tcgen05_persist_c64_loadb_bn64"}
KERNEL_IDS = {v: k for k, v in KERNEL_NAMES.items()}


def tn_autotune(p: Plan, prec: str = "bf16x6", n_bits: int = 0, stream=None) -> list:
    """Time every kernel that supports each contraction step and keep the fastest (stored in the
    plan for ``prec``). Returns the chosen kernel names, one per step."""
    k = np.zeros(max(p.info["n_steps"], 1), dtype=np.int32)
    _check(LIB.tn_autotune(p.ptr, PRECISIONS[prec], int(n_bits), _stream_handle(stream),
                           k.ctypes.data_as(C.POINTER(C.c_int32))))
    return [KERNEL_NAMES.get(int(x), str(int(x))) for x in k[: p.info["n_steps"]]]


def tn_plan_kernels(p: Plan, prec: str = "bf16x6") -> list:
    k = np.zeros(max(p.info["n_steps"], 1), dtype=np.int32)
    _check(LIB.tn_plan_kernels(p.ptr, PRECISIONS[prec], k.ctypes.data_as(C.POINTER(C.c_int32))))
    return [KERNEL_NAMES.get(int(x), str(int(x))) for x in k[: p.info["n_steps"]]]


def tn_plan_set_kernels(p: Plan, prec: str, kernels=None):
    """Force the step kernels (names or ids, one per step); None returns to the shape heuristic."""
    if kernels is None:
        _check(LIB.tn_plan_set_kernels(p.ptr, PRECISIONS[prec], None))
        return
    k = np.asarray([KERNEL_IDS[x] if isinstance(x, str) else int(x) for x in kernels], dtype=np.int32)
    if len(k) != p.info["n_steps"]:
        raise ValueError(f"need {p.info['n_steps']} kernels, got {len(k)}")
    _check(LIB.tn_plan_set_kernels(p.ptr, PRECISIONS[prec], k.ctypes.data_as(C.POINTER(C.c_int32))))


def _packed_concat(plans, bits_list):
    rows, counts = [], []
    for p, b in zip(plans, bits_list):
        n = p.circuit.n_qubits
        words = max((n + 63) // 64, 1)
        b = np.asarray(b)
        if b.dtype != np.uint64 or b.ndim != 2 or b.shape[1] != words:
            b = pack_bits(b.reshape(-1, n))
        rows.append(np.ascontiguousarray(b).reshape(-1))
        counts.append(b.shape[0])
    return np.ascontiguousarray(np.concatenate(rows)), np.asarray(counts, dtype=np.int64)


class Batch:
    """Several circuits' amplitudes as one CUDA graph launch (tn_batch_*)."""

    def __init__(self, ptr, plans, counts, prec):
        self.ptr = ptr
        self.plans = list(plans)      # plans (and their circuits) outlive the batch
        self.counts = counts
        self.prec = prec

    def __del__(self):
        if getattr(self, "ptr", None) and LIB is not None:
            LIB.tn_batch_free(self.ptr)
            self.ptr = None

    @property
    def total(self) -> int:
        return int(self.counts.sum())

    def split(self, flat):
        """Per-circuit views of a concatenated result array."""
        return np.split(flat, np.cumsum(self.counts)[:-1])


def tn_batch_create(plans, bits_list, prec: str = "bf16x6", hbm_budget_bytes: float = 0.0, stream=None) -> Batch:
    """``bits_list[i]``: circuit i's bitstrings ((B_i, n_i) 0/1 or packed uint64 words);
    ``hbm_budget_bytes``: bound on all circuits' workspaces together (0: none)."""
    flat, counts = _packed_concat(plans, bits_list)
    arr = (C.c_void_p * len(plans))(*[p.ptr for p in plans])
    out = C.c_void_p()
    _check(LIB.tn_batch_create(arr, len(plans), C.c_void_p(flat.ctypes.data),
                               counts.ctypes.data_as(C.POINTER(C.c_int64)), PRECISIONS[prec],
                               float(hbm_budget_bytes), _stream_handle(stream), C.byref(out)))
    return Batch(out.value, plans, counts, prec)


def tn_batch_set_bits(b: Batch, bits, stream=None):
    """``bits``: the concatenated packed words (numpy uint64, or a torch tensor, host or device),
    or a list of per-circuit bitstring arrays."""
    if isinstance(bits, (list, tuple)):
        bits, _ = _packed_concat(b.plans, bits)
    ptr = bits.data_ptr() if hasattr(bits, "data_ptr") else np.ascontiguousarray(bits).ctypes.data
    _check(LIB.tn_batch_set_bits(b.ptr, C.c_void_p(ptr), _stream_handle(stream)))


def tn_batch_run(b: Batch, stream=None):
    _check(LIB.tn_batch_run(b.ptr, _stream_handle(stream)))


def tn_batch_read(b: Batch, out=None, stream=None):
    """All amplitudes concatenated in plan order (numpy complex128), or into ``out`` (a torch
    complex128 tensor, host or device)."""
    res = np.zeros(b.total, dtype=np.complex128) if out is None else out
    optr = res.ctypes.data if isinstance(res, np.ndarray) else res.data_ptr()
    _check(LIB.tn_batch_read(b.ptr, C.c_void_p(optr), _stream_handle(stream)))
    return res


def tn_batch_info(b: Batch) -> dict:
    k, m = C.c_int64(), C.c_int64()
    _check(LIB.tn_batch_info(b.ptr, C.byref(k), C.byref(m)))
    return {"graph_kernels": k.value, "device_bytes": m.value}


def tn_batch_free(b: Batch):
    if b.ptr:
        LIB.tn_batch_free(b.ptr)
        b.ptr = None


def tn_build_largest_chi(n_qubits: int, edges, gates, split_cycle: int, chis=(2, 4, 8, 16, 32, 64),
                         max_intermediate: int = 1 << 24, cutoff_rel: float = 1e-12, allocator="torch", stream=None):
    """Circuit, plan and chi for the largest bond cap in ``chis`` whose contraction needs no cut:
    every intermediate of the path at most ``max_intermediate`` elements per bitstring. Raises
    TNError(TN_ERR_NO_PATH) if even the smallest cap needs one."""
    c = tn_build(n_qubits, edges, gates, allocator)
    best = None
    for chi in sorted(chis):
        tn_evolve_two_sided(c, split_cycle, chi, cutoff_rel, stream)
        p = tn_path(c, max_intermediate=max_intermediate)
        if p.info["n_slices"] > 1:
            break
        best = chi
        del p
    if best is None:
        raise TNError(TN_ERR_NO_PATH, f"no cap in {tuple(chis)} fits {max_intermediate} elements without cuts")
    tn_evolve_two_sided(c, split_cycle, best, cutoff_rel, stream)
    return c, tn_path(c, max_intermediate=max_intermediate), best

"""Python driver of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU baseline leg
of the benchmark load it; the library's contraction path never does. It
imports nothing from the CUDA path -- circuits arrive as gate lists from the
seeded input generator, plans as (qubit, segment) keys.

Functions
  build()                   compile liboracle.so with gcc (-fopenmp)
  statevector(circ)         brute-force C|0^n> (complex128, index sum_q x_q 2^q)
  free_vars(circ)           free variable keys (qubit, segment) of the network
  graph_edges(circ)         edges of the free-variable graph (indices into free_vars)
  contract(circ, bits, order=None, mu=(), slices=None, per_slice=False, counts=False)
                            sliced bucket elimination (Eq. 2, 4, 5) in FP64
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles oracle.c into oracle/_build/liboracle.so (plain C99, -O2, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=gnu99", "-O2", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(L):
    P = ctypes.POINTER
    i32p, f64p, u8p = P(ctypes.c_int), P(ctypes.c_double), P(ctypes.c_uint8)
    gate_args = [ctypes.c_int, ctypes.c_size_t, i32p, i32p, i32p, f64p]
    L.orc_statevector.argtypes = gate_args + [f64p]
    L.orc_network_vars.argtypes = gate_args + [i32p, i32p, ctypes.c_int]
    L.orc_network_graph.argtypes = gate_args + [i32p, ctypes.c_int]
    L.orc_contract.argtypes = gate_args + [
        u8p, i32p, i32p, ctypes.c_int, i32p, i32p, ctypes.c_int,
        ctypes.c_uint64, ctypes.c_uint64, f64p, f64p, f64p]
    L.orc_num_threads.restype = ctypes.c_int
    return L


class use_library:
    """Context manager: run the oracle functions on another build of oracle.c
    (the tests use it to check that planted mistakes are caught)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _load()
        _lib = _bind(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _gate_arrays(circ):
    g = circ.gates
    kind = np.array([x.kind for x in g] or [0], dtype=np.int32)
    q0 = np.array([x.q0 for x in g] or [0], dtype=np.int32)
    q1 = np.array([x.q1 for x in g] or [0], dtype=np.int32)
    mats = np.zeros((max(len(g), 1), 8), dtype=np.float64)
    for i, x in enumerate(g):
        if x.m:
            mats[i, :] = x.m
    return (circ.n_qubits, len(g), _ptr(kind, ctypes.c_int), _ptr(q0, ctypes.c_int),
            _ptr(q1, ctypes.c_int), _ptr(mats, ctypes.c_double)), (kind, q0, q1, mats)


def num_threads() -> int:
    return _load().orc_num_threads()


def statevector(circ) -> np.ndarray:
    lib = _load()
    args, keep = _gate_arrays(circ)
    out = np.zeros(2 << circ.n_qubits, dtype=np.float64)
    rc = lib.orc_statevector(*args, _ptr(out, ctypes.c_double))
    if rc:
        raise ValueError(f"orc_statevector failed ({rc})")
    return out.view(np.complex128)


def free_vars(circ):
    lib = _load()
    args, keep = _gate_arrays(circ)
    cap = 1 << 16
    qa = np.zeros(cap, dtype=np.int32)
    sa = np.zeros(cap, dtype=np.int32)
    n = lib.orc_network_vars(*args, _ptr(qa, ctypes.c_int), _ptr(sa, ctypes.c_int), cap)
    if n < 0:
        raise ValueError("bad circuit")
    return [(int(qa[i]), int(sa[i])) for i in range(n)]


def graph_edges(circ):
    lib = _load()
    args, keep = _gate_arrays(circ)
    cap = 1 << 20
    e = np.zeros(2 * cap, dtype=np.int32)
    n = lib.orc_network_graph(*args, _ptr(e, ctypes.c_int), cap)
    if n < 0:
        raise ValueError("bad circuit")
    return [(int(e[2 * i]), int(e[2 * i + 1])) for i in range(n)]


def contract(circ, bits, order=None, mu=(), slices=None, per_slice=False, counts=False):
    """FP64 sliced bucket elimination.

    order: list of (qubit, segment) keys of the non-sliced free variables
    (None = the oracle's own min-degree order). mu: list of sliced keys;
    bit j of slice s is mu[j]'s value. slices: (begin, end), default all 2^p.
    Returns the complex sum over the slices, plus the per-slice values and the
    operation counts (complex multiplications, complex additions) if asked.
    """
    lib = _load()
    args, keep = _gate_arrays(circ)
    b = np.ascontiguousarray(np.array(bits, dtype=np.uint8))
    if b.size != circ.n_qubits:
        raise ValueError("bitstring length")
    p = len(mu)
    muq = np.array([k[0] for k in mu] or [0], dtype=np.int32)
    mus = np.array([k[1] for k in mu] or [0], dtype=np.int32)
    if order is None:
        n_order = -1
        oq = np.zeros(1, dtype=np.int32)
        os_ = np.zeros(1, dtype=np.int32)
    else:
        n_order = len(order)
        oq = np.array([k[0] for k in order] or [0], dtype=np.int32)
        os_ = np.array([k[1] for k in order] or [0], dtype=np.int32)
    s0, s1 = slices if slices is not None else (0, 1 << p)
    total = np.zeros(2, dtype=np.float64)
    per = np.zeros(2 * max(s1 - s0, 1), dtype=np.float64)
    cnt = np.zeros(2, dtype=np.float64)
    rc = lib.orc_contract(*args, _ptr(b, ctypes.c_uint8), _ptr(oq, ctypes.c_int), _ptr(os_, ctypes.c_int),
                          n_order, _ptr(muq, ctypes.c_int), _ptr(mus, ctypes.c_int), p,
                          s0, s1, _ptr(total, ctypes.c_double), _ptr(per, ctypes.c_double),
                          _ptr(cnt, ctypes.c_double))
    if rc:
        raise ValueError(f"orc_contract failed ({rc})")
    amp = complex(total[0], total[1])
    out = [amp]
    if per_slice:
        out.append(per[: 2 * (s1 - s0)].view(np.complex128).copy())
    if counts:
        out.append((float(cnt[0]), float(cnt[1])))
    return out[0] if len(out) == 1 else tuple(out)

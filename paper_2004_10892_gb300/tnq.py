"""Thin Python binding of the tnq C-ABI (include/tnq.h): argument marshalling only.

Every step of planning and contraction runs in the native library
(libtnq.so: host C++ planner + sm_103a CUDA kernels). PyTorch is used only to
allocate the device workspace and to pass the current CUDA stream. If the
library is missing, every call raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("TNQ_LIB", os.path.join(_HERE, "_build", "libtnq.so"))
_lib = None

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(6)
SLICER_TREE_TRIMMING, SLICER_DEGREE, SLICER_DIRECT, SLICER_LEARNED, SLICER_BETWEENNESS = range(5)
PREC_C64, PREC_SPLIT_BF16, PREC_SPLIT_TF32 = range(3)
ORDER_MIN_FILL, ORDER_MIN_DEGREE = range(2)


class TnqError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"tnq status {status}: {msg}")
        self.status = status


class Gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("m", ctypes.c_double * 8)]


class PlanOpts(ctypes.Structure):
    _fields_ = [("slicer", ctypes.c_int32), ("max_bag_log2", ctypes.c_int32), ("min_p", ctypes.c_int32),
                ("max_p", ctypes.c_int32), ("seed", ctypes.c_uint64), ("precision", ctypes.c_int32),
                ("gemm_min_k_log2", ctypes.c_int32), ("ordering", ctypes.c_int32),
                ("td_rebuild", ctypes.c_int32), ("fuse_min_rank", ctypes.c_int32), ("leaf_absorb", ctypes.c_int32),
                ("reorder_every", ctypes.c_int32), ("order_trials", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_free_vars", ctypes.c_int32),
                ("n_leaf_tensors", ctypes.c_int32), ("n_buckets", ctypes.c_int32), ("p", ctypes.c_int32),
                ("tau_full", ctypes.c_int32), ("tau", ctypes.c_int32), ("max_bag", ctypes.c_int32),
                ("n_slices", ctypes.c_uint64), ("flops_per_slice", ctypes.c_double),
                ("bytes_per_slice", ctypes.c_double), ("peak_bytes_per_slice", ctypes.c_double),
                ("total_flops", ctypes.c_double), ("n_gemm_buckets", ctypes.c_int32),
                ("n_fused_groups", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


# Every function the header declares: name -> (restype, argtypes)
_P = ctypes.POINTER
_i32p, _f64p, _u8p, _szp = _P(ctypes.c_int32), _P(ctypes.c_double), _P(ctypes.c_uint8), _P(ctypes.c_size_t)
_vp = ctypes.c_void_p
SIGNATURES = {
    "tnq_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "tnq_last_error": (ctypes.c_char_p, []),
    "tnq_version": (ctypes.c_char_p, []),
    "tnq_plan_opts_default": (None, [_P(PlanOpts)]),
    "tnq_plan_from_circuit": (ctypes.c_int, [ctypes.c_int32, _P(Gate), ctypes.c_size_t, _P(PlanOpts), _P(_vp)]),
    "tnq_plan_from_network": (ctypes.c_int, [ctypes.c_int32, _i32p, ctypes.c_size_t, _P(ctypes.c_int64), _i32p,
                                             _f64p, _P(PlanOpts), _P(_vp)]),
    "tnq_plan_destroy": (None, [_vp]),
    "tnq_plan_info_get": (ctypes.c_int, [_vp, _P(PlanInfo)]),
    "tnq_plan_order": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "tnq_plan_sliced": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "tnq_plan_buckets": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p]),
    "tnq_plan_workspace_bytes": (ctypes.c_size_t, [_vp, ctypes.c_uint32]),
    "tnq_contract_sliced": (ctypes.c_int, [_vp, _u8p, ctypes.c_uint64, ctypes.c_uint64, _vp, ctypes.c_size_t,
                                           ctypes.c_uint32, _vp, _f64p, _f64p]),
    "tnq_plan_autotune": (ctypes.c_int, [_vp, _u8p, _vp, ctypes.c_size_t, ctypes.c_uint32, _vp, _i32p]),
    "tnq_contract_sliced_noalloc": (ctypes.c_int, [_vp, _u8p, ctypes.c_uint64, ctypes.c_uint64, _vp, _f64p, _f64p]),
    "tnq_amplitudes_batch": (ctypes.c_int, [_P(_vp), ctypes.c_size_t, _u8p, _szp, _vp, ctypes.c_size_t, _vp,
                                            _f64p]),
    "tnq_learned_features": (ctypes.c_int32, []),
    "tnq_learned_param_count": (ctypes.c_size_t, [ctypes.c_int32]),
    "tnq_learned_set_weights": (ctypes.c_int, [_P(ctypes.c_float), ctypes.c_int32]),
    "tnq_learned_dataset": (ctypes.c_int, [ctypes.c_int32, _P(Gate), ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32,
                                           _P(ctypes.c_float), _P(ctypes.c_float), _i32p, _i32p,
                                           ctypes.c_size_t, _szp]),
    "tnq_learned_predict_host": (ctypes.c_int, [_P(ctypes.c_float), ctypes.c_int32, _P(ctypes.c_float),
                                                ctypes.c_size_t, _P(ctypes.c_float)]),
    "tnq_mlp_workspace_floats": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_size_t]),
    "tnq_mlp_forward": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, ctypes.c_size_t, _vp, _vp, _vp]),
    "tnq_mlp_backward": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_size_t, _vp, _vp, _vp, _vp]),
    "tnq_mlp_sgd": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_size_t, ctypes.c_float, ctypes.c_float, _vp]),
    "tnq_graph_treewidth": (ctypes.c_int, [ctypes.c_int32, ctypes.c_size_t, _i32p, _i32p, _i32p, _i32p]),
    "tnq_graph_order": (ctypes.c_int, [ctypes.c_int32, ctypes.c_size_t, _i32p, ctypes.c_int32, _i32p]),
    "tnq_graph_tree_decomposition": (ctypes.c_int, [ctypes.c_int32, ctypes.c_size_t, _i32p, _i32p, ctypes.c_int32,
                                                    ctypes.c_int32, _i32p, _i32p, _i32p, _i32p]),
    "tnq_graph_greedy_deletion": (ctypes.c_int, [ctypes.c_int32, ctypes.c_size_t, _i32p, _i32p, ctypes.c_int32,
                                                 ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p]),
    "tnq_graph_betweenness": (ctypes.c_int, [ctypes.c_int32, ctypes.c_size_t, _i32p, _f64p]),
    "tnq_plan_fused_chains": (ctypes.c_int, [_vp, _i32p, ctypes.c_size_t, _szp]),
    "tnq_plan_keep_chains": (ctypes.c_int, [_vp, _i32p, ctypes.c_size_t]),
    "tnq_plan_tuning": (ctypes.c_int, [_vp, _i32p, _i32p]),
    "tnq_plan_set_tuning": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32]),
    "tnq_circuit_graph": (ctypes.c_int, [ctypes.c_int32, _P(Gate), ctypes.c_size_t, ctypes.c_size_t, _i32p, _szp, _i32p]),
}


def lib():
    """Loads libtnq.so (raises if it was not built; there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtnq.so not found at {LIB_PATH}: run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            if not hasattr(L, name):
                continue
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != OK:
        raise TnqError(status, lib().tnq_last_error().decode())


def _ptr(a, ct):
    return a.ctypes.data_as(_P(ct))


def default_opts(**kw) -> PlanOpts:
    o = PlanOpts()
    lib().tnq_plan_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def gates_array(circ):
    arr = (Gate * max(len(circ.gates), 1))()
    for i, g in enumerate(circ.gates):
        arr[i].kind = g.kind
        arr[i].q0 = g.q0
        arr[i].q1 = g.q1
        if g.m:
            for j in range(8):
                arr[i].m[j] = g.m[j]
    return arr


class Plan:
    """A compiled plan (tnq_plan_from_circuit). Frees itself when collected."""

    def __init__(self, circ, **opts):
        self.n_qubits = circ.n_qubits
        o = default_opts(**opts)
        arr = gates_array(circ)
        h = _vp()
        _check(lib().tnq_plan_from_circuit(circ.n_qubits, arr, len(circ.gates), ctypes.byref(o), ctypes.byref(h)))
        self.handle = h

    @classmethod
    def from_network(cls, dims, tensors, **opts):
        """tnq_plan_from_network: a closed network with L-valued indices.
        tensors: list of (index tuple, complex array of shape (dims[i] for i in
        the tuple)); the arrays are passed in C order."""
        self = cls.__new__(cls)
        self.n_qubits = 0
        o = default_opts(**opts)
        d = np.ascontiguousarray(np.array(list(dims) or [1], dtype=np.int32))
        offs = [0]
        idx = []
        data = []
        for ind, arr in tensors:
            idx.extend(int(i) for i in ind)
            offs.append(len(idx))
            data.append(np.ascontiguousarray(np.asarray(arr, dtype=np.complex128)).reshape(-1))
        off = np.array(offs, dtype=np.int64)
        ia = np.ascontiguousarray(np.array(idx or [0], dtype=np.int32))
        da = np.ascontiguousarray(np.concatenate(data) if data else np.zeros(1, np.complex128)).view(np.float64)
        h = _vp()
        _check(lib().tnq_plan_from_network(len(dims), _ptr(d, ctypes.c_int32), len(tensors), _ptr(off, ctypes.c_int64),
                                           _ptr(ia, ctypes.c_int32), _ptr(da, ctypes.c_double), ctypes.byref(o),
                                           ctypes.byref(h)))
        self.handle = h
        return self

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.tnq_plan_destroy(h)
            self.handle = None

    def info(self) -> dict:
        inf = PlanInfo()
        _check(lib().tnq_plan_info_get(self.handle, ctypes.byref(inf)))
        return inf.as_dict()

    def order(self):
        n = self.info()["n_buckets"]
        q = np.zeros(max(n, 1), np.int32)
        s = np.zeros(max(n, 1), np.int32)
        _check(lib().tnq_plan_order(self.handle, _ptr(q, ctypes.c_int32), _ptr(s, ctypes.c_int32)))
        return [(int(q[i]), int(s[i])) for i in range(n)]

    def sliced(self):
        p = self.info()["p"]
        q = np.zeros(max(p, 1), np.int32)
        s = np.zeros(max(p, 1), np.int32)
        _check(lib().tnq_plan_sliced(self.handle, _ptr(q, ctypes.c_int32), _ptr(s, ctypes.c_int32)))
        return [(int(q[i]), int(s[i])) for i in range(p)]

    def buckets(self):
        n = self.info()["n_buckets"]
        bag = np.zeros(max(n, 1), np.int32)
        k = np.zeros(max(n, 1), np.int32)
        gm = np.zeros(max(n, 1), np.int32)
        _check(lib().tnq_plan_buckets(self.handle, _ptr(bag, ctypes.c_int32), _ptr(k, ctypes.c_int32),
                                      _ptr(gm, ctypes.c_int32)))
        return bag[:n].copy(), k[:n].copy(), gm[:n].copy()

    def fused_chains(self):
        """Last-bucket indices of the chains this plan runs fused (tnq_plan_fused_chains)."""
        n = ctypes.c_size_t()
        _check(lib().tnq_plan_fused_chains(self.handle, None, 0, ctypes.byref(n)))
        out = np.zeros(max(n.value, 1), np.int32)
        _check(lib().tnq_plan_fused_chains(self.handle, _ptr(out, ctypes.c_int32), n.value, ctypes.byref(n)))
        return [int(x) for x in out[: n.value]]

    def keep_chains(self, last_buckets):
        """Keep fused only the listed chains (tnq_plan_keep_chains)."""
        arr = np.ascontiguousarray(np.array(list(last_buckets) or [0], dtype=np.int32))
        _check(lib().tnq_plan_keep_chains(self.handle, _ptr(arr, ctypes.c_int32), len(last_buckets)))

    def tuning(self):
        """(gemm_min_k_log2, tile_low) the program is compiled with (tnq_plan_tuning)."""
        k, t = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().tnq_plan_tuning(self.handle, ctypes.byref(k), ctypes.byref(t)))
        return k.value, t.value

    def set_tuning(self, gemm_min_k_log2: int, tile_low: int):
        """Recompile with the given GEMM cut-over and tile shape (tnq_plan_set_tuning)."""
        _check(lib().tnq_plan_set_tuning(self.handle, gemm_min_k_log2, tile_low))

    def workspace_bytes(self, batch: int = 1) -> int:
        return int(lib().tnq_plan_workspace_bytes(self.handle, batch))

    def autotune(self, bits, workspace=None, max_batch: int = 0, stream=None) -> int:
        """tnq_plan_autotune: keep each fused chain only where it measures faster. Returns #chains fused."""
        import torch

        b = _bits_array(bits, self.n_qubits)
        if workspace is None:
            workspace = torch.empty(self.workspace_bytes(max(max_batch, 1)), dtype=torch.uint8, device="cuda")
        n = ctypes.c_int32()
        _check(lib().tnq_plan_autotune(self.handle, _ptr(b, ctypes.c_uint8), ctypes.c_void_p(workspace.data_ptr()),
                                       workspace.numel(), max_batch, _stream_ptr(stream), ctypes.byref(n)))
        return n.value


def _bits_array(bits, n):
    if bits is None and n == 0:  # a general network has no qubits
        return np.zeros(1, np.uint8)
    b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8))
    if b.size != n:
        raise ValueError(f"bitstring has {b.size} entries, plan has {n} qubits")
    return b


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def default_workspace_bytes(plans, want_items: int, fraction: float = 0.5) -> int:
    """Bytes of workspace for the largest power-of-two batch of at most
    want_items that fits every plan in `fraction` of the free device memory."""
    import torch

    free, _ = torch.cuda.mem_get_info()
    budget = int(free * fraction)
    batch = 1
    while batch * 2 <= max(want_items, 1) and max(p.workspace_bytes(batch * 2) for p in plans) <= budget:
        batch *= 2
    return max(p.workspace_bytes(batch) for p in plans) if plans else 256


def default_workspace(plans, want_items: int, fraction: float = 0.5):
    """A device workspace (torch uint8) of default_workspace_bytes."""
    import torch

    return torch.empty(default_workspace_bytes(plans, want_items, fraction), dtype=torch.uint8, device="cuda")


def contract_sliced(plan: Plan, bits=None, slice_begin: int = 0, slice_end: int | None = None, workspace=None,
                    max_batch: int = 0, stream=None, per_slice: bool = False):
    """tnq_contract_sliced: FP64 partial sum over slices [begin, end) (Eq. 5).

    workspace: a CUDA torch tensor (uint8) or None to allocate one with torch.
    Returns the complex sum, plus the per-slice values if per_slice.
    """
    import torch

    n_slices = plan.info()["n_slices"]
    if slice_end is None:
        slice_end = n_slices
    b = _bits_array(bits, plan.n_qubits)
    if workspace is None:
        want = max_batch if max_batch > 0 else min(slice_end - slice_begin, 1 << 16) or 1
        workspace = default_workspace([plan], want)
    out = np.zeros(2, np.float64)
    per = np.zeros(2 * max(slice_end - slice_begin, 1), np.float64) if per_slice else None
    _check(lib().tnq_contract_sliced(plan.handle, _ptr(b, ctypes.c_uint8), slice_begin, slice_end,
                                     ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), max_batch,
                                     _stream_ptr(stream), _ptr(out, ctypes.c_double),
                                     _ptr(per, ctypes.c_double) if per is not None else None))
    amp = complex(out[0], out[1])
    if per_slice:
        return amp, per[: 2 * (slice_end - slice_begin)].view(np.complex128).copy()
    return amp


def contract_sliced_noalloc(plan: Plan, bits=None, slice_begin: int = 0, slice_end: int | None = None, stream=None,
                            per_slice: bool = False):
    """tnq_contract_sliced_noalloc: as contract_sliced, with the library's static
    device scratch instead of a workspace (no device allocation anywhere)."""
    n_slices = plan.info()["n_slices"]
    if slice_end is None:
        slice_end = n_slices
    b = _bits_array(bits, plan.n_qubits)
    out = np.zeros(2, np.float64)
    per = np.zeros(2 * max(slice_end - slice_begin, 1), np.float64) if per_slice else None
    _check(lib().tnq_contract_sliced_noalloc(plan.handle, _ptr(b, ctypes.c_uint8), slice_begin, slice_end,
                                             _stream_ptr(stream), _ptr(out, ctypes.c_double),
                                             _ptr(per, ctypes.c_double) if per is not None else None))
    amp = complex(out[0], out[1])
    if per_slice:
        return amp, per[: 2 * (slice_end - slice_begin)].view(np.complex128).copy()
    return amp


def amplitudes_batch(plans, bitstrings, workspace=None, stream=None):
    """tnq_amplitudes_batch: plans[i] gets the bitstrings bitstrings[i] (a list of bit lists)."""
    import torch

    flat = []
    offs = [0]
    for p, bl in zip(plans, bitstrings):
        for bits in bl:
            flat.append(_bits_array(bits, p.n_qubits))
        offs.append(offs[-1] + len(bl))
    allbits = np.concatenate(flat) if flat else np.zeros(1, np.uint8)
    offsets = np.array(offs, dtype=np.uint64).astype(np.uintp)
    handles = (ctypes.c_void_p * max(len(plans), 1))(*[p.handle for p in plans])
    if workspace is None:
        import torch

        want = max([(1 << p.info()["p"]) * len(b) for p, b in zip(plans, bitstrings)] or [1])
        lanes = min(4, len({id(p) for p, b in zip(plans, bitstrings) if len(b)}) or 1)
        one = default_workspace_bytes(plans, want, fraction=0.5 / lanes)
        # one share per concurrent lane, plus the call's staging area and accumulators
        workspace = torch.empty(lanes * one + 32 * offs[-1] + (1 << 20), dtype=torch.uint8, device="cuda")
    out = np.zeros(2 * max(offs[-1], 1), np.float64)
    _check(lib().tnq_amplitudes_batch(handles, len(plans), _ptr(allbits, ctypes.c_uint8),
                                      offsets.ctypes.data_as(_P(ctypes.c_size_t)),
                                      ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                      _stream_ptr(stream), _ptr(out, ctypes.c_double)))
    return out[: 2 * offs[-1]].view(np.complex128).copy()


# ---- graph-level planning ------------------------------------------------------
def _edges_array(edges):
    e = np.ascontiguousarray(np.array(edges, dtype=np.int32).reshape(-1)) if len(edges) else np.zeros(2, np.int32)
    return e, len(edges)


def graph_treewidth(n, edges, order, bag_sizes=False):
    """Algorithm 1; with bag_sizes=True also the per-step bag sizes |N(u)|+1."""
    e, ne = _edges_array(edges)
    o = np.ascontiguousarray(np.array(order, dtype=np.int32)) if n else np.zeros(1, np.int32)
    tau = ctypes.c_int32()
    sizes = np.zeros(max(n, 1), np.int32)
    _check(lib().tnq_graph_treewidth(n, ne, _ptr(e, ctypes.c_int32), _ptr(o, ctypes.c_int32), ctypes.byref(tau),
                                     _ptr(sizes, ctypes.c_int32)))
    return (tau.value, [int(x) for x in sizes[:n]]) if bag_sizes else tau.value


def graph_order(n, edges, method=ORDER_MIN_FILL):
    e, ne = _edges_array(edges)
    o = np.zeros(max(n, 1), np.int32)
    _check(lib().tnq_graph_order(n, ne, _ptr(e, ctypes.c_int32), method, _ptr(o, ctypes.c_int32)))
    return [int(x) for x in o[:n]]


def graph_tree_decomposition(n, edges, order):
    e, ne = _edges_array(edges)
    o = np.ascontiguousarray(np.array(order, dtype=np.int32)) if n else np.zeros(1, np.int32)
    cap_b, cap_v = max(n, 1), max(n * n, 1)
    nb = ctypes.c_int32()
    offs = np.zeros(cap_b + 1, np.int32)
    verts = np.zeros(cap_v, np.int32)
    par = np.zeros(cap_b, np.int32)
    _check(lib().tnq_graph_tree_decomposition(n, ne, _ptr(e, ctypes.c_int32), _ptr(o, ctypes.c_int32), cap_b, cap_v,
                                              ctypes.byref(nb), _ptr(offs, ctypes.c_int32),
                                              _ptr(verts, ctypes.c_int32), _ptr(par, ctypes.c_int32)))
    bags = [[int(v) for v in verts[offs[b]:offs[b + 1]]] for b in range(nb.value)]
    return bags, [int(x) for x in par[: nb.value]]


def graph_greedy_deletion(n, edges, order, m, slicer=SLICER_TREE_TRIMMING, seed=0, td_rebuild=False,
                          reorder_every=0):
    e, ne = _edges_array(edges)
    o = np.ascontiguousarray(np.array(order, dtype=np.int32)) if n else np.zeros(1, np.int32)
    mu = np.zeros(max(m, 1), np.int32)
    tau = np.zeros(max(m, 1), np.int32)
    _check(lib().tnq_graph_greedy_deletion(n, ne, _ptr(e, ctypes.c_int32), _ptr(o, ctypes.c_int32), m, slicer, seed,
                                           int(td_rebuild), int(reorder_every), _ptr(mu, ctypes.c_int32),
                                           _ptr(tau, ctypes.c_int32)))
    return [int(x) for x in mu[:m]], [int(x) for x in tau[:m]]


def graph_betweenness(n, edges):
    """Betweenness centrality of every vertex (tnq_graph_betweenness)."""
    e, ne = _edges_array(edges)
    out = np.zeros(max(n, 1), np.float64)
    _check(lib().tnq_graph_betweenness(n, ne, _ptr(e, ctypes.c_int32), _ptr(out, ctypes.c_double)))
    return out[:n]


def circuit_graph(circ):
    """(n_vertices, edges) of the circuit's free-variable graph (tnq_circuit_graph)."""
    arr = gates_array(circ)
    n = ctypes.c_int32()
    ne = ctypes.c_size_t()
    L = lib()
    rc = L.tnq_circuit_graph(circ.n_qubits, arr, len(circ.gates), 0, ctypes.byref(n), ctypes.byref(ne), None)
    if rc != OK and ne.value == 0:
        _check(rc)
    e = np.zeros(2 * max(ne.value, 1), np.int32)
    _check(L.tnq_circuit_graph(circ.n_qubits, arr, len(circ.gates), ne.value, ctypes.byref(n), ctypes.byref(ne),
                               _ptr(e, ctypes.c_int32)))
    return n.value, e[:2 * ne.value].reshape(-1, 2)

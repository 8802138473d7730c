"""Learned slicing proposer: data generation, GPU training, weights.

Data come from the plain heuristic itself (tnq_learned_dataset: candidates of
each tree-trimming step with their exact cost change). The network is trained
on the GPU with the library's own kernels (tnq_mlp_backward / tnq_mlp_sgd);
the planner runs it on the host (TNQ_SLICER_LEARNED) after
tnq_learned_set_weights, falling back to tree-trimming without weights.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import tnq

HIDDEN = 128
TRAINED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "proposer_h128.npy")


def features() -> int:
    return int(tnq.lib().tnq_learned_features())


def param_count(hidden: int = HIDDEN) -> int:
    return int(tnq.lib().tnq_learned_param_count(hidden))


def dataset(circ, max_steps: int = 12, ordering: int = tnq.ORDER_MIN_FILL, with_candidates: bool = False):
    """(features [n, F], labels [n], step [n]) of one circuit (+ candidate ids)."""
    L = tnq.lib()
    F = features()
    arr = tnq.gates_array(circ)
    cap = 1 << 14
    while True:
        X = np.zeros((cap, F), np.float32)
        y = np.zeros(cap, np.float32)
        st = np.zeros(cap, np.int32)
        cd = np.zeros(cap, np.int32)
        n = ctypes.c_size_t()
        rc = L.tnq_learned_dataset(circ.n_qubits, arr, len(circ.gates), ordering, max_steps,
                                   X.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                   y.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                   st.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   cd.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), cap, ctypes.byref(n))
        if rc == tnq.OK:
            out = (X[: n.value], y[: n.value], st[: n.value])
            return out + (cd[: n.value],) if with_candidates else out
        if n.value > cap:
            cap = n.value
            continue
        tnq._check(rc)


def init_params(seed: int = 0, hidden: int = HIDDEN) -> np.ndarray:
    """He-initialised weights, zero biases (numpy, FP32)."""
    F = features()
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal((hidden, F)) * np.sqrt(2.0 / F), np.zeros(hidden),
             rng.standard_normal((hidden, hidden)) * np.sqrt(2.0 / hidden), np.zeros(hidden),
             rng.standard_normal(hidden) * np.sqrt(1.0 / hidden), np.zeros(1)]
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


def gpu_forward(params, X, hidden: int = HIDDEN, stream=None):
    """Forward pass with the library's GPU kernels (torch CUDA tensors in/out)."""
    import torch

    L = tnq.lib()
    n = X.shape[0]
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    work = torch.empty(L.tnq_mlp_workspace_floats(hidden, n), dtype=torch.float32, device="cuda")
    tnq._check(L.tnq_mlp_forward(_dptr(params), hidden, _dptr(X), n, _dptr(out), _dptr(work),
                                 tnq._stream_ptr(stream)))
    return out


def gpu_grad(params, X, y, hidden: int = HIDDEN, stream=None):
    """(loss, gradient) with the library's GPU backward kernel."""
    import torch

    L = tnq.lib()
    n = X.shape[0]
    grads = torch.empty_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    work = torch.empty(L.tnq_mlp_workspace_floats(hidden, n), dtype=torch.float32, device="cuda")
    tnq._check(L.tnq_mlp_backward(_dptr(params), hidden, _dptr(X), _dptr(y), n, _dptr(grads), _dptr(loss),
                                  _dptr(work), tnq._stream_ptr(stream)))
    return loss, grads


def train(X, y, epochs: int = 200, batch: int = 1024, lr: float = 0.05, mu: float = 0.9, seed: int = 0,
          hidden: int = HIDDEN):
    """Mini-batch SGD with momentum on the GPU; returns (weights numpy, loss history)."""
    import torch

    L = tnq.lib()
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y, np.float32)).cuda()
    params = torch.from_numpy(init_params(seed, hidden)).cuda()
    mom = torch.zeros_like(params)
    grads = torch.empty_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    n = Xd.shape[0]
    b = min(batch, n)
    work = torch.empty(L.tnq_mlp_workspace_floats(hidden, b), dtype=torch.float32, device="cuda")
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    st = tnq._stream_ptr(None)
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).cuda()
        tot = 0.0
        for i in range(0, n - b + 1, b):
            idx = perm[i:i + b]
            xb = Xd.index_select(0, idx).contiguous()
            yb = yd.index_select(0, idx).contiguous()
            tnq._check(L.tnq_mlp_backward(_dptr(params), hidden, _dptr(xb), _dptr(yb), b, _dptr(grads), _dptr(loss),
                                          _dptr(work), st))
            tnq._check(L.tnq_mlp_sgd(_dptr(params), _dptr(grads), _dptr(mom), params.numel(), lr, mu, st))
            tot += float(loss)
        hist.append(tot / max(1, n // b))
    return params.cpu().numpy(), hist


def load_trained():
    """Weights trained by train_proposer.py on the 500-circuit set (numpy, FP32)."""
    return np.load(TRAINED)


def set_weights(params, hidden: int = HIDDEN):
    """Installs weights for TNQ_SLICER_LEARNED (None clears them)."""
    L = tnq.lib()
    if params is None:
        tnq._check(L.tnq_learned_set_weights(None, 0))
        return
    p = np.ascontiguousarray(params, np.float32)
    tnq._check(L.tnq_learned_set_weights(p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), hidden))


def predict_host(params, X, hidden: int = HIDDEN):
    L = tnq.lib()
    p = np.ascontiguousarray(params, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    out = np.zeros(X.shape[0], np.float32)
    P = ctypes.POINTER(ctypes.c_float)
    tnq._check(L.tnq_learned_predict_host(p.ctypes.data_as(P), hidden, X.ctypes.data_as(P), X.shape[0],
                                          out.ctypes.data_as(P)))
    return out

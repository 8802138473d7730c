"""Split-precision tensor-core GEMM (tcgen05) against FP64 matrix products."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
BF16, TF32 = 0, 1


def tc_gemm(tnq_lib, kind, A, B):
    L = tnq_lib.lib()
    f = L.tnq_internal_gemm_selftest
    P = ctypes.POINTER
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_float),
                  P(ctypes.c_float), P(ctypes.c_float), ctypes.c_char_p, ctypes.c_size_t]
    batch, M, K = A.shape
    N = B.shape[1]
    A = np.ascontiguousarray(A, np.float32)
    B = np.ascontiguousarray(B, np.float32)
    C = np.zeros((batch, M, N), np.float32)
    msg = ctypes.create_string_buffer(256)
    rc = f(kind, batch, M, N, K, A.ctypes.data_as(P(ctypes.c_float)), B.ctypes.data_as(P(ctypes.c_float)),
           C.ctypes.data_as(P(ctypes.c_float)), msg, 256)
    assert rc == 0, msg.value
    return C


@pytest.mark.parametrize("kind", [BF16, TF32])
def test_exact_small_integers(cuda, tnq_lib, kind):
    """Small integers are exact in BF16/TF32 and in FP32 sums: any layout or
    descriptor mistake shows as a nonzero difference."""
    rng = np.random.default_rng(1)
    A = rng.integers(-3, 4, size=(2, 256, 128)).astype(np.float32)
    B = rng.integers(-3, 4, size=(2, 128, 128)).astype(np.float32)
    C = tc_gemm(tnq_lib, kind, A, B)
    ref = np.einsum("bmk,bnk->bmn", A.astype(np.float64), B.astype(np.float64))
    assert np.array_equal(C, ref.astype(np.float32))


@pytest.mark.parametrize("kind,tol", [(BF16, 3e-5), (TF32, 3e-6)])
def test_split_precision_accuracy(cuda, tnq_lib, kind, tol):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((3, 128, 256)).astype(np.float32)
    B = rng.standard_normal((3, 256, 256)).astype(np.float32)
    C = tc_gemm(tnq_lib, kind, A, B)
    ref = np.einsum("bmk,bnk->bmn", A.astype(np.float64), B.astype(np.float64))
    err = np.max(np.abs(C - ref)) / np.max(np.abs(ref))
    assert err < tol, err


def test_bounded_wait_reports_timeout(cuda, tnq_lib):
    """A device wait that can never complete gives up after its limit and the
    host reads TNQ_ETIMEOUT; the context stays usable afterwards."""
    import time

    L = tnq_lib.lib()
    f = L.tnq_internal_wait_timeout_selftest
    f.argtypes = [ctypes.c_ulonglong]
    t = time.perf_counter()
    assert f(200_000_000) == tnq_lib.ETIMEOUT
    assert time.perf_counter() - t < 10
    A = np.ones((1, 128, 64), np.float32)
    C = tc_gemm(tnq_lib, BF16, A, A)
    assert np.all(C == 64)


def _gemm_forms(tnq_lib, plan, mode, batch):
    L = tnq_lib.lib()
    f = L.tnq_internal_gemm_forms
    P = ctypes.POINTER
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, P(ctypes.c_int32), ctypes.c_int, P(ctypes.c_int32)]
    buf = (ctypes.c_int32 * 256)()
    n = ctypes.c_int32()
    assert f(plan.handle, mode, batch, buf, 256, ctypes.byref(n)) == 0
    return [buf[i] for i in range(n.value)]


@pytest.mark.parametrize("case", ["7x7-24", "6x6-24"])
def test_fused_a_gemm_matches_packed_form_and_oracle(cuda, tnq_lib, oracle_lib, monkeypatch, case):
    """GEMM steps whose A operand is read, scaled and split inside the GEMM
    kernel (fused-A form; here with K of 2^3..2^6 values, so partly zero-filled
    K steps, item-dependent and item-invariant operands) against the same plan
    with every operand packed first, and every slice against the oracle at the
    split-precision tolerance."""
    from paper_2004_10892_gb300 import inputs as I

    if case == "7x7-24":
        circ, bits = I.random_grid_circuit(7, 7, 24, 1), I.random_bitstring(49, 1)
        kw, tuning = dict(max_bag_log2=20, max_p=30, reorder_every=1, precision=1, gemm_min_k_log2=4), (3, 64)
    else:
        circ, bits = I.random_grid_circuit(6, 6, 24, 7), I.random_bitstring(36, 7)
        kw, tuning = dict(max_bag_log2=20, max_p=20, reorder_every=1, precision=1, gemm_min_k_log2=4,
                          fuse_min_rank=10), (4, 64)
    n = circ.n_qubits
    plan = tnq_lib.Plan(circ, **kw)
    plan.set_tuning(*tuning)
    n_sl = plan.info()["n_slices"]
    assert 1 in _gemm_forms(tnq_lib, plan, 0, n_sl)
    amp, per = tnq_lib.contract_sliced(plan, bits, per_slice=True)
    monkeypatch.setenv("TNQ_GEMM_FUSED_A", "0")
    packed = tnq_lib.Plan(circ, **kw)
    packed.set_tuning(*tuning)
    assert set(_gemm_forms(tnq_lib, packed, 0, n_sl)) == {0}
    amp0, per0 = tnq_lib.contract_sliced(packed, bits, per_slice=True)
    monkeypatch.delenv("TNQ_GEMM_FUSED_A")
    scale = np.abs(per0).max()
    assert np.max(np.abs(per - per0)) <= 1e-5 * scale
    ref, ref_per = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced(), per_slice=True)
    floor = 2.0 ** (-n / 2) / np.sqrt(len(per))
    for s in range(len(per)):
        den = max(abs(ref_per[s]), floor)
        assert abs(per[s] - ref_per[s]) / den < 1e-4, (s, per[s], ref_per[s])
    assert abs(amp - ref) / max(abs(ref), 2.0 ** (-n / 2)) < 1e-4

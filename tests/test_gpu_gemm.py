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

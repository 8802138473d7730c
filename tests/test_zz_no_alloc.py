"""tnq_contract_sliced_noalloc: the allocation-free entry point.

It serves callers that cannot allocate device memory (their pool allocator
already holds all the device memory they may use, or cudaMalloc's implicit
synchronisation is not affordable in their loop): its scratch is a fixed
64 MiB static device array instead of a caller workspace. Each case compares
it with the workspace entry point and with the FP64 oracle, on two calls in a
row (the array keeps the previous call's contents). This file is collected
last so that a run stopping at the first failure has run every other test
before it.
"""
import ctypes

import numpy as np
import pytest

from paper_2004_10892_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-5
SPLIT_TOL = 1e-4


def rel_err(a, ref, n):
    floor = 2.0 ** (-n / 2)
    den = abs(ref) if abs(ref) ** 2 >= floor ** 2 / 10 else floor
    return abs(a - ref) / den


def test_noalloc_matches_workspace_entry_point_and_oracle(cuda, tnq_lib, oracle_lib):
    circ = I.random_grid_circuit(5, 5, 20, 2)
    bits = I.random_bitstring(25, 2)
    plan = tnq_lib.Plan(circ, min_p=4, max_p=4)
    ref_amp, ref_per = tnq_lib.contract_sliced(plan, bits, per_slice=True)
    o_amp, o_per = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced(), per_slice=True)
    scale = np.abs(ref_per).max()
    for call in range(2):  # the array keeps the previous call's contents
        amp, per = tnq_lib.contract_sliced_noalloc(plan, bits, per_slice=True)
        assert abs(amp - ref_amp) <= TOL * abs(ref_amp), (call, amp, ref_amp)
        assert np.max(np.abs(per - ref_per)) <= TOL * scale, call
        assert rel_err(amp, o_amp, 25) < TOL, (call, amp, o_amp)
        for s in range(len(per)):
            assert rel_err(per[s], o_per[s], 25) < TOL, (call, s)
        part = tnq_lib.contract_sliced_noalloc(plan, bits, 3, 11)
        assert abs(part - ref_per[3:11].sum()) <= TOL * np.abs(ref_per[3:11]).sum()
        assert abs(part - o_per[3:11].sum()) <= TOL * np.abs(o_per[3:11]).sum()


def test_noalloc_second_plan_after_first(cuda, tnq_lib, oracle_lib):
    """A different plan right after: nothing stale from the previous call leaks in."""
    for seed in (3, 4):
        circ = I.random_grid_circuit(4, 4, 16, seed)
        plan = tnq_lib.Plan(circ, min_p=2, max_p=2)
        bits = I.random_bitstring(16, seed)
        ref = tnq_lib.contract_sliced(plan, bits)
        o_ref = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced())
        for _ in range(2):
            got = tnq_lib.contract_sliced_noalloc(plan, bits)
            assert abs(got - ref) <= TOL * abs(ref)
            assert rel_err(got, o_ref, 16) < TOL


def _step_kinds(tnq_lib, plan):
    L = tnq_lib.lib()
    P = ctypes.POINTER(ctypes.c_int32)
    k = np.zeros(4096, np.int32)
    n = ctypes.c_int32()
    assert L.tnq_internal_step_kinds(plan.handle, 0, 1, k.ctypes.data_as(P), None, 4096, ctypes.byref(n)) == 0
    t = np.zeros(4096, np.int32)
    m = ctypes.c_int32()
    assert L.tnq_internal_group_tails(plan.handle, 0, 1, t.ctypes.data_as(P), 4096, ctypes.byref(m)) == 0
    return k[: n.value], t[: m.value]


def test_noalloc_split_precision_gemm_and_register_tail_steps(cuda, tnq_lib, oracle_lib):
    """A 3xBF16 plan whose slices run tensor-core GEMM steps (operand and pack
    scratch inside the static array), fused chains with a register tail and
    early-bucket level launches; per-slice values against the workspace entry
    point and the oracle at the split-precision tolerance."""
    circ = I.random_grid_circuit(5, 6, 24, 0)
    bits = I.random_bitstring(30, 0)
    plan = tnq_lib.Plan(circ, max_bag_log2=18, min_p=3, max_p=30, precision=1, gemm_min_k_log2=3,
                        fuse_min_rank=8, reorder_every=1)
    kinds, tails = _step_kinds(tnq_lib, plan)
    assert (kinds == 2).sum() >= 1, "no GEMM step in the plan"
    assert (tails > 0).sum() >= 1, "no register-tail chain in the plan"
    ref_amp, ref_per = tnq_lib.contract_sliced(plan, bits, per_slice=True)
    o_amp, o_per = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced(), per_slice=True)
    for call in range(2):
        amp, per = tnq_lib.contract_sliced_noalloc(plan, bits, per_slice=True)
        assert np.max(np.abs(per - ref_per)) <= 1e-6 * np.abs(ref_per).max(), call
        for s in range(len(per)):
            assert rel_err(per[s], o_per[s], 30) < SPLIT_TOL, (call, s, per[s], o_per[s])
        assert rel_err(amp, o_amp, 30) < SPLIT_TOL


def test_noalloc_allocates_no_device_memory(cuda, tnq_lib):
    """After a first call (address lookup, host tables), further calls leave the
    device's free memory unchanged."""
    import torch

    circ = I.random_grid_circuit(5, 5, 20, 6)
    bits = I.random_bitstring(25, 6)
    plan = tnq_lib.Plan(circ, min_p=3, max_p=3, precision=1, gemm_min_k_log2=3, fuse_min_rank=8)
    first = tnq_lib.contract_sliced_noalloc(plan, bits)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert tnq_lib.contract_sliced_noalloc(plan, bits) == first
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_plans_beyond_the_scratch(cuda, tnq_lib):
    circ = I.random_grid_circuit(7, 7, 32, 0)
    plan = tnq_lib.Plan(circ, min_p=2, max_p=2)  # one slice needs GBs
    assert plan.workspace_bytes(1) > 64 << 20
    with pytest.raises(tnq_lib.TnqError) as e:
        tnq_lib.contract_sliced_noalloc(plan, I.random_bitstring(49, 0), 0, 1)
    assert e.value.status == tnq_lib.ENOMEM
    assert "static scratch" in str(e.value)

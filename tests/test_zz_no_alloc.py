"""tnq_contract_sliced_noalloc: the allocation-free entry point.

It serves callers that cannot allocate device memory (their pool allocator
already holds the memory they may use, another thread keeps a stream capture
open, or cudaMalloc's implicit synchronisation is not affordable): its scratch
is a fixed 64 MiB static device array instead of a caller workspace. This
file is collected last so that a run stopping at the first failure has run
every other test before it.
"""
import numpy as np
import pytest

from paper_2004_10892_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-5


def test_noalloc_matches_workspace_entry_point(cuda, tnq_lib):
    circ = I.random_grid_circuit(5, 5, 20, 2)
    bits = I.random_bitstring(25, 2)
    plan = tnq_lib.Plan(circ, min_p=4, max_p=4)
    ref_amp, ref_per = tnq_lib.contract_sliced(plan, bits, per_slice=True)
    scale = np.abs(ref_per).max()
    for call in range(2):  # the array keeps the previous call's contents
        amp, per = tnq_lib.contract_sliced_noalloc(plan, bits, per_slice=True)
        assert abs(amp - ref_amp) <= TOL * abs(ref_amp), (call, amp, ref_amp)
        assert np.max(np.abs(per - ref_per)) <= TOL * scale, call
        part = tnq_lib.contract_sliced_noalloc(plan, bits, 3, 11)
        assert abs(part - ref_per[3:11].sum()) <= TOL * np.abs(ref_per[3:11]).sum()


def test_noalloc_second_plan_after_first(cuda, tnq_lib):
    """A different plan right after: nothing stale from the previous call leaks in."""
    for seed in (3, 4):
        circ = I.random_grid_circuit(4, 4, 16, seed)
        plan = tnq_lib.Plan(circ, min_p=2, max_p=2)
        bits = I.random_bitstring(16, seed)
        ref = tnq_lib.contract_sliced(plan, bits)
        for _ in range(2):
            got = tnq_lib.contract_sliced_noalloc(plan, bits)
            assert abs(got - ref) <= TOL * abs(ref)


def test_noalloc_rejects_plans_beyond_the_scratch(cuda, tnq_lib):
    circ = I.random_grid_circuit(7, 7, 32, 0)
    plan = tnq_lib.Plan(circ, min_p=2, max_p=2)  # one slice needs GBs
    assert plan.workspace_bytes(1) > 64 << 20
    with pytest.raises(tnq_lib.TnqError) as e:
        tnq_lib.contract_sliced_noalloc(plan, I.random_bitstring(49, 0), 0, 1)
    assert e.value.status == tnq_lib.ENOMEM
    assert "static scratch" in str(e.value)

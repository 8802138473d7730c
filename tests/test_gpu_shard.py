"""Slice sharding through the CUDA path (Section II.D: the 2^p sub-contractions
of Eq. 4 are independent, Eq. 5 sums them): shard.sharded_amplitude and the
checkpointed partial sums with tnq_contract_sliced as the contraction call,
against the whole-range call and the FP64 oracle. Two gloo ranks share the one
GPU as independent processes (their kernels never wait on each other; the only
exchange is the host-side all-reduce of one complex128)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2004_10892_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _case():
    circ = I.random_grid_circuit(5, 5, 20, 8)
    bits = I.random_bitstring(25, 8)
    return circ, bits


def _plan(tnq_lib, circ):
    return tnq_lib.Plan(circ, min_p=5, max_p=5)


def test_sharded_amplitude_world_one_with_checkpoint(cuda, tnq_lib, oracle_lib, tmp_path):
    from paper_2004_10892_gb300.shard import Checkpoint, contract_range, sharded_amplitude, slice_range

    circ, bits = _case()
    plan = _plan(tnq_lib, circ)
    n_sl = plan.info()["n_slices"]
    calls = []

    def contract(b, e):
        calls.append((b, e))
        return tnq_lib.contract_sliced(plan, bits, b, e)

    whole = tnq_lib.contract_sliced(plan, bits)
    ref = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced())
    amp = sharded_amplitude(contract, n_sl, chunk=4)
    assert len(calls) == n_sl // 4
    assert abs(amp - whole) <= 1e-12 * abs(whole) + 1e-300
    assert abs(amp - ref) <= TOL * abs(ref)
    # the ranges of a world of 3, contracted one after another, sum to the amplitude
    parts = [contract_range(contract, *slice_range(n_sl, r, 3), chunk=3) for r in range(3)]
    assert abs(sum(parts) - ref) <= TOL * abs(ref)
    # checkpointed partial sums: a restart contracts only the missing chunks
    path = str(tmp_path / "ck.json")
    calls.clear()
    first = contract_range(contract, 0, n_sl // 2, chunk=4, checkpoint=Checkpoint(path, "5x5-s8"))
    assert len(calls) == n_sl // 8
    calls.clear()
    total = contract_range(contract, 0, n_sl, chunk=4, checkpoint=Checkpoint(path, "5x5-s8"))
    assert calls == [(b, b + 4) for b in range(n_sl // 2, n_sl, 4)]
    assert abs(total - ref) <= TOL * abs(ref)
    assert abs(first - tnq_lib.contract_sliced(plan, bits, 0, n_sl // 2)) <= 1e-12 * abs(first)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, outdir):
    import datetime

    import torch
    import torch.distributed as dist

    from paper_2004_10892_gb300 import tnq
    from paper_2004_10892_gb300.shard import sharded_amplitude

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    try:
        torch.cuda.set_device(0)
        circ, bits = _case()
        plan = tnq.Plan(circ, min_p=5, max_p=5)
        amp = sharded_amplitude(lambda b, e: tnq.contract_sliced(plan, bits, b, e), plan.info()["n_slices"], chunk=2)
        with open(os.path.join(outdir, f"r{rank}.txt"), "w") as f:
            f.write(f"{amp.real!r} {amp.imag!r}")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_on_the_gpu_sum_to_the_amplitude(cuda, tnq_lib, oracle_lib, tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    circ, bits = _case()
    plan = _plan(tnq_lib, circ)
    ref = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced())
    got = []
    for r in range(2):
        re, im = map(float, open(tmp_path / f"r{r}.txt").read().split())
        got.append(complex(re, im))
    assert got[0] == got[1]
    assert abs(got[0] - ref) <= TOL * abs(ref)
    assert np.isfinite(got[0].real)

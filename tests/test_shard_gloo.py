"""Multi-process slice sharding on CPU: world size 2 over gloo.

Each rank contracts its contiguous slice range with the FP64 oracle (the
stand-in for the GPU call on a CPU-only machine); the all-reduced partial
sums equal the unsliced amplitude (Eq. 5). Failure handling is exercised on
the host: a rank that dies before the exchange makes the other one fail
with an error instead of hanging, and a restarted rank resumes from its
checkpoint.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2004_10892_gb300 import inputs as I
from paper_2004_10892_gb300.shard import Checkpoint, contract_range, slice_range


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _circuit():
    circ = I.random_grid_circuit(3, 4, 12, 6)
    bits = I.random_bitstring(12, 6)
    return circ, bits


def _keys(circ):
    from oracle import oracle

    fv = oracle.free_vars(circ)
    mu = [fv[2], fv[7], fv[11]]
    return [v for v in fv if v not in mu], mu


def _worker(rank, world, port, outdir, mode):
    import torch.distributed as dist

    from oracle import oracle
    from paper_2004_10892_gb300.shard import sharded_amplitude

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import datetime

    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    circ, bits = _circuit()
    order, mu = _keys(circ)

    def contract(b, e):
        return oracle.contract(circ, bits, order=order, mu=mu, slices=(b, e))

    try:
        if mode == "die" and rank == 1:
            os._exit(3)  # a rank that never reaches the exchange
        amp = sharded_amplitude(contract, 1 << len(mu), chunk=1)
        with open(os.path.join(outdir, f"r{rank}.txt"), "w") as f:
            f.write(f"{amp.real!r} {amp.imag!r}")
    except Exception as exc:  # the survivor sees an error, not a hang
        with open(os.path.join(outdir, f"r{rank}.err"), "w") as f:
            f.write(type(exc).__name__)
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def test_slice_range_partition():
    for n in (0, 1, 7, 8, 256, 1000):
        for world in (1, 2, 3, 8):
            ranges = [slice_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slice_range(8, 2, 2)


def test_two_ranks_sum_to_unsliced_amplitude(oracle_lib, tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path), "ok"), nprocs=2, join=True, start_method="spawn")
    circ, bits = _circuit()
    ref = oracle_lib.contract(circ, bits)
    for r in range(2):
        re, im = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert abs(complex(re, im) - ref) < 1e-12


def test_dead_rank_fails_the_exchange(oracle_lib, tmp_path):
    port = _free_port()
    ctx = mp.start_processes(_worker, args=(2, port, str(tmp_path), "die"), nprocs=2, join=False,
                             start_method="spawn")
    for p in ctx.processes:
        p.join(120)
        assert not p.is_alive()
    assert (tmp_path / "r0.err").exists() and not (tmp_path / "r0.txt").exists()


def test_checkpoint_resume(oracle_lib, tmp_path):
    circ, bits = _circuit()
    order, mu = _keys(circ)
    calls = []

    def contract(b, e):
        calls.append((b, e))
        return oracle_lib.contract(circ, bits, order=order, mu=mu, slices=(b, e))

    path = str(tmp_path / "ck.json")
    ck = Checkpoint(path, "plan-A")
    part = contract_range(contract, 0, 4, chunk=1, checkpoint=ck)
    assert len(calls) == 4
    # a restart finds the four chunks done and only contracts the rest
    calls.clear()
    ck2 = Checkpoint(path, "plan-A")
    total = contract_range(contract, 0, 8, chunk=1, checkpoint=ck2)
    assert calls == [(4, 5), (5, 6), (6, 7), (7, 8)]
    assert abs(total - oracle_lib.contract(circ, bits)) < 1e-12
    assert abs(part - sum(oracle_lib.contract(circ, bits, order=order, mu=mu, slices=(s, s + 1)) for s in range(4))) < 1e-12
    # another plan's checkpoint is ignored
    assert Checkpoint(path, "plan-B").done == []

"""Slice sharding across processes (Section II.D: the 2^p sub-contractions of
Eq. 4 are independent; Eq. 5 sums them).

Each rank contracts a contiguous range of slices with the C-ABI call
``tnq_contract_sliced`` (or any function with its signature) and the FP64
partial sums are combined with one all-reduce of a complex128 -- the only
exchange this path has. A checkpoint records the finished ranges and their
partial sums so a restarted job contracts only what is missing.
"""
from __future__ import annotations

import json
import os


def slice_range(n_slices: int, rank: int, world: int):
    """Contiguous, balanced [begin, end) of the slices owned by `rank`."""
    if world < 1 or not 0 <= rank < world or n_slices < 0:
        raise ValueError("bad rank/world/n_slices")
    base, extra = divmod(n_slices, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


class Checkpoint:
    """Finished slice ranges with their FP64 partial sums, keyed by a plan tag.

    The file is JSON: {"tag": ..., "done": [[begin, end, re, im], ...]}; it is
    rewritten atomically after every finished chunk.
    """

    def __init__(self, path: str, tag: str):
        self.path, self.tag = path, tag
        self.done = []
        if path and os.path.exists(path):
            with open(path) as f:
                d = json.load(f)
            if d.get("tag") == tag:
                self.done = [tuple(x) for x in d.get("done", [])]

    def covered(self, begin: int, end: int):
        """Finished sub-ranges inside [begin, end), sorted."""
        return sorted((b, e, re, im) for b, e, re, im in self.done if b >= begin and e <= end)

    def add(self, begin: int, end: int, value: complex):
        self.done.append((begin, end, value.real, value.imag))
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump({"tag": self.tag, "done": self.done}, f)
            os.replace(tmp, self.path)


def contract_range(contract, begin: int, end: int, chunk: int = 0, checkpoint: Checkpoint | None = None) -> complex:
    """Sum of slices [begin, end) via contract(b, e) -> complex, in chunks of
    `chunk` slices (0 = one call), skipping chunks a checkpoint already has.
    Partial sums are added in increasing slice order."""
    step = chunk if chunk > 0 else max(end - begin, 1)
    done = {(b, e): complex(re, im) for b, e, re, im in (checkpoint.covered(begin, end) if checkpoint else [])}
    total = 0j
    for b in range(begin, end, step):
        e = min(end, b + step)
        if (b, e) in done:
            total += done[(b, e)]
            continue
        v = contract(b, e)
        if checkpoint is not None:
            checkpoint.add(b, e, v)
        total += v
    return total


def sharded_amplitude(contract, n_slices: int, group=None, chunk: int = 0, checkpoint: Checkpoint | None = None):
    """Amplitude = all-reduce over ranks of each rank's partial sum (Eq. 5).

    contract(begin, end) -> complex is the rank's sub-contraction call. With no
    process group (or world size 1) the sum stays local.
    """
    import torch
    import torch.distributed as dist

    if group is not None or (dist.is_available() and dist.is_initialized()):
        rank, world = dist.get_rank(group), dist.get_world_size(group)
    else:
        rank, world = 0, 1
    b, e = slice_range(n_slices, rank, world)
    part = contract_range(contract, b, e, chunk, checkpoint) if e > b else 0j
    if world == 1:
        return part
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([part.real, part.imag], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return complex(float(t[0]), float(t[1]))

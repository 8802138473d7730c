"""Trains the learned slicing proposer and compares it with tree-trimming.

  python -m paper_2004_10892_gb300.train_proposer [--circuits 500] [--epochs 40]
         [--out paper_2004_10892_gb300/data/proposer_h128.npy] [--measure]

Training data: seeded random grid circuits, 5x5..8x8, depths 1+20+1..1+40+1;
for each, the candidates of up to 12 tree-trimming steps with their exact
cost change (tnq_learned_dataset). Training: mini-batch SGD on the GPU with
the library's own forward/backward/SGD kernels. Evaluation: the 8x8 depth
1+32+1 circuit sliced by tree-trimming and by the learned proposer, at equal
p and at equal bag limit, compared by the exact cost model (total flops,
per-slice traffic) and, with --measure, by measured contraction time per
slice on the GPU. Prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import inputs, learned, tnq

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "data", "proposer_h128.npy")


def training_circuits(n: int, seed: int = 1000):
    rng = inputs.SplitMix64(seed)
    out = []
    for i in range(n):
        side = 5 + rng.below(4)           # 5..8
        depth = 20 + 4 * rng.below(6)     # 20..40
        out.append(inputs.random_grid_circuit(side, side, depth, seed + i))
    return out


def build_dataset(circuits, max_steps: int = 12):
    Xs, ys = [], []
    for c in circuits:
        X, y, _ = learned.dataset(c, max_steps=max_steps)
        Xs.append(X)
        ys.append(y)
    return np.concatenate(Xs), np.concatenate(ys)


def plan_pair(circ, weights, **kw):
    tt = tnq.Plan(circ, slicer=tnq.SLICER_TREE_TRIMMING, **kw)
    learned.set_weights(weights)
    try:
        ln = tnq.Plan(circ, slicer=tnq.SLICER_LEARNED, **kw)
    finally:
        learned.set_weights(None)
    return tt, ln


def summary(plan):
    i = plan.info()
    return {"p": i["p"], "tau": i["tau"], "max_bag": i["max_bag"], "total_flops": i["total_flops"],
            "log2_total_flops": float(np.log2(i["total_flops"])), "bytes_per_slice": i["bytes_per_slice"]}


def measure_per_slice(plan, bits, n_sample: int = 32):
    """Seconds per slice, contracting slices [0, n_sample) at once on the GPU."""
    import torch

    n = min(n_sample, plan.info()["n_slices"])
    ws = torch.empty(plan.workspace_bytes(n), dtype=torch.uint8, device="cuda")
    tnq.contract_sliced(plan, bits, 0, n, workspace=ws, max_batch=n)
    torch.cuda.synchronize()
    t = time.perf_counter()
    tnq.contract_sliced(plan, bits, 0, n, workspace=ws, max_batch=n)
    torch.cuda.synchronize()
    return (time.perf_counter() - t) / n


def evaluate(weights, measure: bool = False):
    circ = inputs.random_grid_circuit(8, 8, 32, 0)
    bits = inputs.random_bitstring(64, 0)
    res = {"circuit": "grid 8x8 depth 1+32+1 seed 0", "equal_p": [], "equal_bag": []}
    for p in (8, 11, 13):
        tt, ln = plan_pair(circ, weights, min_p=p, max_p=p)
        res["equal_p"].append({"p": p, "tree_trimming": summary(tt), "learned": summary(ln)})
    for mb in (30, 28):
        tt, ln = plan_pair(circ, weights, max_bag_log2=mb, max_p=60)
        row = {"max_bag_log2": mb, "tree_trimming": summary(tt), "learned": summary(ln)}
        if measure:
            for name, pl in (("tree_trimming", tt), ("learned", ln)):
                s = measure_per_slice(pl, bits)
                row[name]["measured_s_per_slice"] = s
                row[name]["measured_s_per_amplitude"] = s * pl.info()["n_slices"]
        res["equal_bag"].append(row)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--circuits", type=int, default=500)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--measure", action="store_true")
    args = ap.parse_args()
    t0 = time.perf_counter()
    X, y = build_dataset(training_circuits(args.circuits))
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    w, hist = learned.train(X, y, epochs=args.epochs, batch=1024, lr=0.02, mu=0.9)
    t_train = time.perf_counter() - t0
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    np.save(args.out, w)
    out = {"rows": int(len(y)), "data_s": t_data, "train_s": t_train, "loss_first": hist[0], "loss_last": hist[-1],
           "weights": os.path.relpath(args.out, os.path.dirname(HERE)), "evaluation": evaluate(w, args.measure)}
    print(json.dumps(out))


if __name__ == "__main__":
    main()

"""Score comparison for the greedy mu-treewidth deletion (Algorithm 2).

  python -m paper_2004_10892_gb300.score_compare [--grids 6x6:24 7x7:32 8x8:32] [--seeds 0 1 2]
         [--m 20] [--scores tree_trimming degree betweenness direct ...] [--out scores.json]

For each seeded random grid circuit (the synthetic stand-ins of Section IV's
Boixo circuits) the free-variable graph is ordered once by the greedy
min-fill heuristic; then each score deletes m vertices one at a time
(Algorithm 2) and the treewidth of the reduced order (Algorithm 1) is
recorded after every deletion, with the wall time of the heuristic. This is
the experiment of Section IV (treewidth against the number of deleted
vertices for the degree, betweenness, direct-reduction and tree-trimming
scores, and their running times), on the host. The "+reorder" rows add
Algorithm 2's optional recomputation: the greedy min-fill order of the
reduced graph is recomputed after every 5 deletions (the paper recomputes a
tree decomposition with an external solver instead). Prints one JSON object and a
summary table of the mean treewidth at a few deletion counts.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs, tnq

# name -> (score, recompute the order after every this many deletions; 0: never)
SCORES = {"tree_trimming": (tnq.SLICER_TREE_TRIMMING, 0), "degree": (tnq.SLICER_DEGREE, 0),
          "betweenness": (tnq.SLICER_BETWEENNESS, 0), "direct": (tnq.SLICER_DIRECT, 0),
          "direct+reorder": (tnq.SLICER_DIRECT, 5), "tree_trimming+reorder": (tnq.SLICER_TREE_TRIMMING, 5)}


def parse_grid(s: str):
    side, depth = s.split(":")
    r, c = side.split("x")
    return int(r), int(c), int(depth)


def compare(circ, m: int, scores):
    n, edges = tnq.circuit_graph(circ)
    order = tnq.graph_order(n, edges, tnq.ORDER_MIN_FILL)
    tau0 = tnq.graph_treewidth(n, edges, order)
    row = {"circuit": circ.name, "vertices": n, "edges": int(len(edges)), "tau0": tau0, "scores": {}}
    for name in scores:
        t = time.perf_counter()
        slicer, reorder = SCORES[name]
        mu, tau = tnq.graph_greedy_deletion(n, edges, order, min(m, n), slicer=slicer, reorder_every=reorder)
        row["scores"][name] = {"tau": tau, "mu": mu, "seconds": time.perf_counter() - t}
    return row


def summary(rows, scores, points):
    lines = ["score                  " + "".join(f"  tau@{p:<3d}" for p in points) + "   seconds"]
    for name in scores:
        cells = []
        for p in points:
            vals = [r["scores"][name]["tau"][p - 1] for r in rows if len(r["scores"][name]["tau"]) >= p]
            cells.append(f"{np.mean(vals):8.2f}" if vals else "      - ")
        secs = np.mean([r["scores"][name]["seconds"] for r in rows])
        lines.append(f"{name:23s}" + "".join(cells) + f"  {secs:8.3f}")
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grids", nargs="+", default=["6x6:24", "7x7:32", "8x8:32"])
    ap.add_argument("--seeds", nargs="+", type=int, default=[0, 1, 2])
    ap.add_argument("--m", type=int, default=20)
    ap.add_argument("--scores", nargs="+", default=list(SCORES), choices=list(SCORES))
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    rows = []
    for g in args.grids:
        r, c, d = parse_grid(g)
        for seed in args.seeds:
            rows.append(compare(inputs.random_grid_circuit(r, c, d, seed), args.m, args.scores))
    points = [p for p in (1, 5, 10, 15, 20, 30, 40) if p <= args.m]
    out = {"m": args.m, "rows": rows, "summary": summary(rows, args.scores, points)}
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f)
    print(out["summary"])


if __name__ == "__main__":
    main()

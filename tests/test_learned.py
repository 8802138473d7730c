"""Learned slicing proposer: labels, host inference, oracle gradients (CPU)."""
import math

import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2004_10892_gb300 import inputs as I


@pytest.fixture(scope="module")
def LN(tnq_lib):
    from paper_2004_10892_gb300 import learned

    return learned


def test_labels_are_exact_cost_changes(tnq_lib, oracle_lib, LN):
    """Step-0 labels recomputed independently: the oracle's own network graph,
    the greedy order and Algorithm 1's bag sizes with the candidate removed."""
    circ = I.random_grid_circuit(5, 5, 16, 2)
    X, y, st, cand = LN.dataset(circ, max_steps=1, with_candidates=True)
    assert len(y) > 0 and np.all(st == 0)
    edges = oracle_lib.graph_edges(circ)
    n = len(oracle_lib.free_vars(circ))
    order = tnq_lib.graph_order(n, edges, 0)
    _, sizes = tnq_lib.graph_treewidth(n, edges, order, bag_sizes=True)
    before = math.log2(sum(2.0 ** r for r in sizes))
    for v, lab in zip(cand, y):
        red = [e for e in edges if v not in e]
        o2 = [u for u in order if u != v] + [v]  # v isolated: its own step costs 2^1, removed below
        _, s2 = tnq_lib.graph_treewidth(n, red, o2, bag_sizes=True)
        after = 1 + math.log2(sum(2.0 ** r for r in s2[:-1]))
        assert abs((after - before) - lab) < 1e-5


def test_host_inference_matches_fp64_oracle(tnq_lib, LN):
    F, H = LN.features(), 32
    rng = np.random.default_rng(0)
    p = (rng.standard_normal(LN.param_count(H)) * 0.3).astype(np.float32)
    X = rng.random((40, F)).astype(np.float32)
    got = LN.predict_host(p, X, H)
    ref, _ = omlp.forward(p, X, F, H)
    assert np.max(np.abs(got - ref)) < 1e-4 * max(1.0, np.max(np.abs(ref)))


def test_oracle_gradient_matches_finite_differences():
    """Pins the FP64 reference backward pass: central differences on every parameter."""
    F, H = 5, 6
    rng = np.random.default_rng(1)
    p = rng.standard_normal(F * H + H + H * H + H + H + 1)
    X = rng.standard_normal((9, F))
    y = rng.standard_normal(9)
    _, g = omlp.loss_and_grad(p, X, y, F, H)
    eps = 1e-6
    fd = np.array([(omlp.loss_only(p + eps * e, X, y, F, H) - omlp.loss_only(p - eps * e, X, y, F, H)) / (2 * eps)
                   for e in np.eye(p.size)])
    assert np.max(np.abs(fd - g)) < 1e-7


def test_learned_slicer_falls_back_without_weights(tnq_lib, LN):
    LN.set_weights(None)
    circ = I.random_grid_circuit(6, 6, 20, 1)
    a = tnq_lib.Plan(circ, slicer=tnq_lib.SLICER_LEARNED, min_p=4, max_p=4)
    b = tnq_lib.Plan(circ, slicer=tnq_lib.SLICER_TREE_TRIMMING, min_p=4, max_p=4)
    assert a.sliced() == b.sliced()


def test_learned_slicer_follows_its_weights(tnq_lib, LN):
    """With weights that score candidates by one feature, the planner deletes
    exactly the candidate a host-side ranking of that feature picks."""
    F, H = LN.features(), 8
    p = np.zeros(LN.param_count(H), np.float32)
    # h1_0 = relu(x[2]) (degree); h2_0 = relu(h1_0); out = -h2_0: prefer the largest degree
    W1 = p[: H * F].reshape(H, F)
    W1[0, 2] = 1.0
    off = H * F + H
    W2 = p[off: off + H * H].reshape(H, H)
    W2[0, 0] = 1.0
    off += H * H + H
    p[off + 0] = -1.0
    LN.set_weights(p, H)
    try:
        circ = I.random_grid_circuit(5, 5, 16, 4)
        plan = tnq_lib.Plan(circ, slicer=tnq_lib.SLICER_LEARNED, min_p=1, max_p=1)
        X, y, st, cand = LN.dataset(circ, max_steps=1, with_candidates=True)
        best = cand[int(np.argmax(X[:, 2]))]
        ties = cand[X[:, 2] == X[:, 2].max()]
        fv_plan = plan.sliced()[0]
        from oracle import oracle

        assert oracle.free_vars(circ).index(fv_plan) in set(int(t) for t in ties)
        assert best in ties
    finally:
        LN.set_weights(None)

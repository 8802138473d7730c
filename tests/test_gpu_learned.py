"""Learned proposer on the GPU: the hand-written forward/backward kernels
against the FP64 oracle network, and a small training run whose planner gain
over tree-trimming is measured on held-out circuits."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2004_10892_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def LN(tnq_lib):
    from paper_2004_10892_gb300 import learned

    return learned


def _data(LN, n=300, seed=0):
    rng = np.random.default_rng(seed)
    F = LN.features()
    return rng.random((n, F)).astype(np.float32), rng.standard_normal(n).astype(np.float32)


@pytest.mark.parametrize("hidden", [16, 128])
def test_gpu_forward_matches_oracle(cuda, LN, hidden):
    import torch

    X, _ = _data(LN)
    p = LN.init_params(3, hidden)
    out = LN.gpu_forward(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(), hidden).cpu().numpy()
    ref, _ = omlp.forward(p, X, LN.features(), hidden)
    assert np.max(np.abs(out - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(out - LN.predict_host(p, X, hidden))) <= 1e-4 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("hidden", [16, 128])
def test_gpu_gradients_match_oracle(cuda, LN, hidden):
    import torch

    X, y = _data(LN, 257, 1)
    p = LN.init_params(5, hidden)
    loss, g = LN.gpu_grad(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), hidden)
    ref_loss, ref_g = omlp.loss_and_grad(p, X, y, LN.features(), hidden)
    g = g.cpu().numpy()
    assert abs(float(loss) - ref_loss) <= 1e-5 * max(1.0, ref_loss)
    assert np.max(np.abs(g - ref_g)) <= 1e-4 * max(1e-3, np.max(np.abs(ref_g)))


def test_training_and_planner_gain(cuda, tnq_lib, LN):
    """Train on 60 small circuits; the learned slicer is then compared with
    tree-trimming on held-out circuits at the same bag limit by exact total
    flops. The learned planner must need fewer total flops on average (a
    negative mean log2 ratio)."""
    from paper_2004_10892_gb300 import train_proposer as TP

    X, y = TP.build_dataset(TP.training_circuits(60, seed=77), max_steps=10)
    w, hist = LN.train(X, y, epochs=30, batch=512, lr=0.02, mu=0.9)
    assert hist[-1] < 0.5 * hist[0]
    deltas = []
    for seed in range(6):
        side = 6 + seed % 2
        circ = I.random_grid_circuit(side, side, 24, 5000 + seed)
        tau = tnq_lib.Plan(circ).info()["tau_full"]
        tt, ln = TP.plan_pair(circ, w, max_bag_log2=tau - 4, max_p=40)
        deltas.append(np.log2(ln.info()["total_flops"]) - np.log2(tt.info()["total_flops"]))
    mean = float(np.mean(deltas))
    print(f"learned vs tree-trimming: mean log2 total-flop ratio {mean:+.3f} over {len(deltas)} circuits {deltas}")
    assert mean < 0.0, deltas

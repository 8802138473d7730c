"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Tolerance: the complex64 path must match the oracle within 1e-5 relative.
The denominator is |a_ref| when |a_ref|^2 >= 2^-n / 10, else 2^-n/2 (an
amplitude far below the Porter-Thomas scale is compared on that scale).
"""
import math

import numpy as np
import pytest

from paper_2004_10892_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel_err(a, ref, n):
    floor = 2.0 ** (-n / 2)
    den = abs(ref) if abs(ref) ** 2 >= floor ** 2 / 10 else floor
    return abs(a - ref) / den


def bits_of(x, n):
    return [(x >> q) & 1 for q in range(n)]


@pytest.mark.parametrize("seed", range(10))
def test_4x4_zero_amplitude(cuda, tnq_lib, oracle_lib, seed):
    """4x4 grid, depth 1+16+1, p = 0: <0^16|C|0^16> vs the oracle and the state vector."""
    circ = I.random_grid_circuit(4, 4, 16, seed)
    plan = tnq_lib.Plan(circ)
    assert plan.info()["p"] == 0
    zero = [0] * 16
    amp = tnq_lib.contract_sliced(plan, zero)
    ref = oracle_lib.contract(circ, zero, order=plan.order(), mu=plan.sliced())
    assert rel_err(amp, ref, 16) < TOL, (amp, ref)
    if seed < 2:
        sv = oracle_lib.statevector(circ)
        assert rel_err(amp, sv[0], 16) < TOL


def test_4x4_full_distribution(cuda, tnq_lib, oracle_lib):
    """All 2^16 amplitudes in one batched call vs the brute-force state vector; norm 1."""
    circ = I.random_grid_circuit(4, 4, 16, 0)
    plan = tnq_lib.Plan(circ)
    sv = oracle_lib.statevector(circ)
    allbits = [bits_of(x, 16) for x in range(1 << 16)]
    amps = tnq_lib.amplitudes_batch([plan], [allbits])
    floor = 2.0 ** -8
    assert np.max(np.abs(amps - sv)) / floor < TOL
    assert abs(np.sum(np.abs(amps) ** 2) - 1.0) < 1e-5


@pytest.mark.parametrize("p", [4, 6, 8])
def test_6x6_sliced_per_slice(cuda, tnq_lib, oracle_lib, p):
    """6x6 grid, depth 1+24+1, p = 4..8: every slice value vs the oracle's."""
    circ = I.random_grid_circuit(6, 6, 24, 0)
    bits = I.random_bitstring(36, 0)
    plan = tnq_lib.Plan(circ, max_bag_log2=24, min_p=p, max_p=p)
    inf = plan.info()
    assert inf["p"] == p and inf["max_bag"] <= 24
    amp, per = tnq_lib.contract_sliced(plan, bits, per_slice=True)
    # the oracle checks a spread of slices one by one, and their sum where cheap
    idx = sorted(set([0, 1, (1 << p) - 1, (1 << p) // 2, 3 % (1 << p)]))
    ref_tot, ref_per = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced(), per_slice=True) \
        if p <= 6 else (None, None)
    for s in idx:
        r = ref_per[s] if ref_per is not None else \
            oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced(), slices=(s, s + 1))
        assert rel_err(per[s], r, 36) < TOL, (s, per[s], r)
    if ref_tot is not None:
        assert rel_err(amp, ref_tot, 36) < TOL
    assert abs(per.sum() - amp) <= 1e-12 * max(abs(amp), 1e-30) + 1e-18


def test_batch_size_does_not_change_slices(cuda, tnq_lib):
    """Every slice is computed by the same arithmetic at any batch size: the
    per-slice values are bit-identical; ragged ranges give the partial sums."""
    circ = I.random_grid_circuit(5, 5, 20, 3)
    bits = I.random_bitstring(25, 3)
    plan = tnq_lib.Plan(circ, min_p=5, max_p=5)
    _, ref = tnq_lib.contract_sliced(plan, bits, per_slice=True)
    for mb in (1, 2, 8, 32):
        _, per = tnq_lib.contract_sliced(plan, bits, max_batch=mb, per_slice=True)
        assert np.array_equal(per, ref), mb
    a, per = tnq_lib.contract_sliced(plan, bits, 3, 27, max_batch=8, per_slice=True)
    assert np.array_equal(per, ref[3:27])
    assert abs(a - ref[3:27].sum()) < 1e-12 * np.abs(ref).sum()


def test_slice_sum_matches_unsliced(cuda, tnq_lib, oracle_lib):
    """Eq. 5 on the GPU: the sum over 2^p slices equals the unsliced oracle amplitude."""
    circ = I.random_grid_circuit(5, 5, 16, 11)
    bits = I.random_bitstring(25, 11)
    plan = tnq_lib.Plan(circ, min_p=3, max_p=3)
    amp = tnq_lib.contract_sliced(plan, bits)
    ref = oracle_lib.contract(circ, bits)
    assert rel_err(amp, ref, 25) < TOL


def test_closed_forms_on_gpu(cuda, tnq_lib):
    # all-H (no free variables): 2^-n/2 for every bitstring
    for n in (1, 5, 30):
        plan = tnq_lib.Plan(I.all_h(n))
        for x in (0, 1, (1 << n) - 1):
            a = tnq_lib.contract_sliced(plan, bits_of(x, n))
            assert abs(a - 2 ** (-n / 2)) < TOL * 2 ** (-n / 2)
    # GHZ and Bell through the batched call
    ghz = tnq_lib.Plan(I.ghz(8), min_p=1, max_p=1)
    bell = tnq_lib.Plan(I.bell())
    ghz_bits = [bits_of(x, 8) for x in (0, 255, 1, 128, 170)]
    bell_bits = [bits_of(x, 2) for x in range(4)]
    out = tnq_lib.amplitudes_batch([ghz, bell], [ghz_bits, bell_bits])
    s = 1 / math.sqrt(2)
    ref = [s, s, 0, 0, 0, s, 0, 0, s]
    assert np.max(np.abs(out - np.array(ref))) < TOL


def test_wire_without_nondiagonal_gate(cuda, tnq_lib, oracle_lib):
    """A qubit whose input segment is its output: <x_q|0> is 0 unless x_q = 0."""
    c = I.Circuit(3, [I.Gate(I.H, 0), I.Gate(I.T, 1), I.Gate(I.CZ, 0, 1), I.Gate(I.H, 2), I.Gate(I.X_1_2, 0)])
    plan = tnq_lib.Plan(c)
    for x in range(8):
        b = bits_of(x, 3)
        a = tnq_lib.contract_sliced(plan, b)
        r = oracle_lib.contract(c, b)
        assert abs(a - r) < TOL


def test_tiny_amplitudes_are_rescaled(cuda, tnq_lib, oracle_lib):
    """Amplitudes far below the FP32 range survive: per-tensor power-of-two exponents."""
    eps = 1e-9
    cth = math.sqrt(1 - eps * eps)
    u = (cth, 0.0, -eps, 0.0, eps, 0.0, cth, 0.0)  # [[c, -e], [e, c]]
    n = 8
    gates = []
    for layer in range(2):
        gates += [I.Gate(I.U1, q, -1, u) for q in range(n)]
        gates += [I.Gate(I.CZ, q, q + 1) for q in range(layer % 2, n - 1, 2)]
    c = I.Circuit(n, gates)
    plan = tnq_lib.Plan(c, min_p=1, max_p=1)
    x = [1, 0, 1, 0, 1, 0, 1, 0]
    a = tnq_lib.contract_sliced(plan, x)
    r = oracle_lib.contract(c, x)
    assert abs(r) < 1e-30
    assert abs(a - r) / abs(r) < TOL


def test_random_small_circuits_all_gates(cuda, tnq_lib, oracle_lib):
    for seed in range(4):
        c = I.random_small_circuit(10, 120, 50 + seed)
        plan = tnq_lib.Plan(c, min_p=2, max_p=2)
        bl = [I.random_bitstring(10, 7 * seed + j) for j in range(4)]
        out = tnq_lib.amplitudes_batch([plan], [bl])
        for b, a in zip(bl, out):
            r = oracle_lib.contract(c, b)
            assert rel_err(a, r, 10) < TOL


def test_uneven_batch_of_plans(cuda, tnq_lib, oracle_lib):
    """Batched serving shape: circuits of different sizes, different bitstring counts."""
    work = I.batched_serving_workload(n_circuits=4, bitstrings_per_circuit=3, seed=5)
    plans, bl = [], []
    for circ, bits in work:
        side = int(round(math.sqrt(circ.n_qubits)))
        plans.append(tnq_lib.Plan(circ, max_bag_log2=18, max_p=16))
        bl.append(bits[: 1 + len(plans) % 3])
    out = tnq_lib.amplitudes_batch(plans, bl)
    k = 0
    for (circ, _), p, bits in zip(work, plans, bl):
        for b in bits:
            if circ.n_qubits <= 36:
                r = oracle_lib.contract(circ, b, order=p.order(), mu=p.sliced())
                assert rel_err(out[k], r, circ.n_qubits) < TOL
            else:
                single = tnq_lib.contract_sliced(p, b)
                assert abs(out[k] - single) <= 1e-9 * abs(single)
            k += 1


@pytest.mark.slow
def test_7x7_full_size_sampled_slices(cuda, tnq_lib, oracle_lib):
    """7x7 grid, depth 1+32+1, per-slice bag <= 28: the benchmark's launch
    configuration (64 slices at once); two slices checked against the oracle,
    the rest through properties (batch-independence of each slice value and the
    slice sum)."""
    import torch

    circ = I.random_grid_circuit(7, 7, 32, 0)
    bits = I.random_bitstring(49, 0)
    plan = tnq_lib.Plan(circ, max_bag_log2=28, max_p=40)
    inf = plan.info()
    assert inf["max_bag"] <= 28
    n_sl = inf["n_slices"]
    B = min(64, n_sl)
    ws = torch.empty(plan.workspace_bytes(B), dtype=torch.uint8, device="cuda")
    amp, per = tnq_lib.contract_sliced(plan, bits, 0, B, workspace=ws, max_batch=B, per_slice=True)
    for s in (0, B - 1):
        r = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced(), slices=(s, s + 1))
        assert abs(per[s] - r) / abs(r) < TOL, (s, per[s], r)
    _, per1 = tnq_lib.contract_sliced(plan, bits, 0, 4, workspace=ws, max_batch=1, per_slice=True)
    assert np.array_equal(per1, per[:4])
    assert abs(per.sum() - amp) <= 1e-12 * np.abs(per).sum()


@pytest.mark.slow
def test_7x7_bench_configuration_every_slice(cuda, tnq_lib, oracle_lib):
    """The benchmark's own configuration at full size: 7x7 depth 1+32+1, order
    recomputed after every deletion, best of 32 randomised greedy orders (p = 5),
    GEMM-shaped chains in 3xBF16, autotuned, all 32 slices in one batch. Every
    slice and the amplitude (Eq. 5: their FP64 sum) against the oracle at the
    split-precision tolerance; cross-slice cancellation is covered because the
    amplitude is compared on its own scale."""
    import torch

    circ = I.random_grid_circuit(7, 7, 32, 0)
    bits = I.random_bitstring(49, 0)
    plan = tnq_lib.Plan(circ, max_bag_log2=28, max_p=40, precision=1, gemm_min_k_log2=4, reorder_every=1,
                        order_trials=32, fuse_min_rank=12)
    inf = plan.info()
    assert inf["max_bag"] <= 28 and inf["n_gemm_buckets"] > 0
    n_sl = inf["n_slices"]
    ws = torch.empty(plan.workspace_bytes(n_sl), dtype=torch.uint8, device="cuda")
    plan.autotune(bits, workspace=ws, max_batch=n_sl)
    amp, per = tnq_lib.contract_sliced(plan, bits, 0, n_sl, workspace=ws, max_batch=n_sl, per_slice=True)
    ref, ref_per = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced(), per_slice=True)
    for s in range(n_sl):
        assert abs(per[s] - ref_per[s]) / abs(ref_per[s]) < SPLIT_TOL, (s, per[s], ref_per[s])
    assert rel_err(amp, ref, 49) < SPLIT_TOL, (amp, ref)
    assert abs(per.sum() - amp) <= 1e-12 * np.abs(per).sum()


@pytest.mark.parametrize("fuse", [1, 4, 8])
def test_fused_chains_match_oracle(cuda, tnq_lib, oracle_lib, fuse):
    """Chains fused into one kernel (down to tiny chains) give the oracle's slices."""
    n_groups = 0
    for seed, (rows, cols, cyc, p) in enumerate([(4, 4, 16, 2), (5, 5, 20, 3), (4, 5, 24, 4)]):
        circ = I.random_grid_circuit(rows, cols, cyc, 20 + seed)
        bits = I.random_bitstring(circ.n_qubits, seed)
        plan = tnq_lib.Plan(circ, min_p=p, max_p=p, fuse_min_rank=fuse)
        n_groups += plan.info()["n_fused_groups"]
        amp, per = tnq_lib.contract_sliced(plan, bits, per_slice=True)
        ref, ref_per = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced(), per_slice=True)
        n = circ.n_qubits
        for s in range(len(per)):
            assert rel_err(per[s], ref_per[s], n) < TOL, (seed, s)
        assert rel_err(amp, ref, n) < TOL
        # batched bitstrings through fused groups
        bl = [I.random_bitstring(n, 100 + j) for j in range(3)]
        out = tnq_lib.amplitudes_batch([plan], [bl])
        for b, a in zip(bl, out):
            assert rel_err(a, oracle_lib.contract(circ, b), n) < TOL
    assert n_groups > 0


def test_fused_equals_unfused(cuda, tnq_lib):
    """Fusion only regroups the same products: slice values agree to FP32 rounding."""
    circ = I.random_grid_circuit(6, 6, 24, 0)
    bits = I.random_bitstring(36, 0)
    fused = tnq_lib.Plan(circ, max_bag_log2=24, min_p=5, max_p=5)
    plain = tnq_lib.Plan(circ, max_bag_log2=24, min_p=5, max_p=5, fuse_min_rank=0)
    assert fused.info()["n_fused_groups"] > 0 and plain.info()["n_fused_groups"] == 0
    assert fused.info()["bytes_per_slice"] < plain.info()["bytes_per_slice"]
    _, a = tnq_lib.contract_sliced(fused, bits, per_slice=True)
    _, b = tnq_lib.contract_sliced(plain, bits, per_slice=True)
    assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(b))


@pytest.mark.parametrize("fuse", [0, 12])
def test_leaf_absorption_matches_oracle(cuda, tnq_lib, oracle_lib, fuse):
    """Gate tensors moved into smaller producing buckets (leaf absorption) give the
    oracle's slices, which keep every gate tensor in the bucket of its earliest
    variable; with absorption off the same plan agrees too."""
    circ = I.random_grid_circuit(6, 6, 24, 2)
    bits = I.random_bitstring(36, 2)
    ref, ref_per = None, None
    for la in (1, 0):
        plan = tnq_lib.Plan(circ, max_bag_log2=22, min_p=5, max_p=5, fuse_min_rank=fuse, leaf_absorb=la)
        amp, per = tnq_lib.contract_sliced(plan, bits, per_slice=True)
        if ref is None:
            ref, ref_per = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced(), per_slice=True)
        for s in range(len(per)):
            assert rel_err(per[s], ref_per[s], 36) < TOL, (la, s)
        assert rel_err(amp, ref, 36) < TOL


def test_autotune_keeps_results(cuda, tnq_lib, oracle_lib):
    """Autotuning only chooses between fused and unfused forms of the same products."""
    circ = I.random_grid_circuit(6, 6, 24, 1)
    bits = I.random_bitstring(36, 1)
    plan = tnq_lib.Plan(circ, max_bag_log2=24, min_p=4, max_p=4, fuse_min_rank=8)
    n0 = plan.info()["n_fused_groups"]
    _, before = tnq_lib.contract_sliced(plan, bits, per_slice=True)
    n1 = plan.autotune(bits, max_batch=16)
    assert 0 <= n1 <= n0 and plan.info()["n_fused_groups"] == n1
    amp, after = tnq_lib.contract_sliced(plan, bits, per_slice=True)
    assert np.max(np.abs(after - before)) <= 1e-6 * np.max(np.abs(before))
    ref = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced())
    assert rel_err(amp, ref, 36) < TOL


SPLIT_TOL = 1e-4


@pytest.mark.parametrize("precision", [1, 2])
def test_split_precision_gemm_buckets_match_oracle(cuda, tnq_lib, oracle_lib, precision):
    """Merged GEMM-shaped buckets on the tensor cores (3xBF16 / 3xTF32) agree
    with the FP64 oracle within the split-precision tolerance."""
    n_gemm = 0
    for seed, (rows, cols, cyc, p) in enumerate([(5, 5, 20, 0), (5, 5, 20, 2), (6, 6, 24, 4)]):
        circ = I.random_grid_circuit(rows, cols, cyc, seed)
        bits = I.random_bitstring(circ.n_qubits, 40 + seed)
        plan = tnq_lib.Plan(circ, min_p=p, max_p=p, precision=precision, gemm_min_k_log2=3)
        n_gemm += plan.info()["n_gemm_buckets"]
        amp, per = tnq_lib.contract_sliced(plan, bits, per_slice=True)
        ref, ref_per = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced(), per_slice=True)
        n = circ.n_qubits
        for s in range(len(per)):
            assert rel_err(per[s], ref_per[s], n) < SPLIT_TOL, (seed, s, per[s], ref_per[s])
        assert rel_err(amp, ref, n) < SPLIT_TOL
        out = tnq_lib.amplitudes_batch([plan], [[bits, I.random_bitstring(n, 99)]])
        assert rel_err(out[0], ref, n) < SPLIT_TOL
    assert n_gemm > 0


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_reordered_plans_match_oracle(cuda, tnq_lib, oracle_lib, precision):
    """Plans whose order is recomputed after every deletion (the bench's 7x7
    configuration) contract to the oracle's slices in complex64 and in both
    split precisions."""
    circ = I.random_grid_circuit(6, 6, 24, 5)
    bits = I.random_bitstring(36, 5)
    plan = tnq_lib.Plan(circ, max_bag_log2=18, max_p=20, reorder_every=1, precision=precision, gemm_min_k_log2=3)
    assert plan.info()["max_bag"] <= 18
    amp, per = tnq_lib.contract_sliced(plan, bits, per_slice=True)
    ref, ref_per = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced(), per_slice=True)
    tol = TOL if precision == 0 else SPLIT_TOL
    for s in range(len(per)):
        assert rel_err(per[s], ref_per[s], 36) < tol, s
    assert rel_err(amp, oracle_lib.contract(circ, bits), 36) < tol


def test_split_precision_agrees_with_c64(cuda, tnq_lib):
    circ = I.random_grid_circuit(6, 6, 24, 3)
    bits = I.random_bitstring(36, 3)
    c64 = tnq_lib.Plan(circ, max_bag_log2=24, min_p=4, max_p=4)
    tf = tnq_lib.Plan(circ, max_bag_log2=24, min_p=4, max_p=4, precision=2, gemm_min_k_log2=3)
    assert tf.info()["n_gemm_buckets"] > 0
    _, a = tnq_lib.contract_sliced(c64, bits, per_slice=True)
    _, b = tnq_lib.contract_sliced(tf, bits, per_slice=True)
    assert np.max(np.abs(a - b)) <= SPLIT_TOL * np.max(np.abs(a))


@pytest.mark.slow
def test_batched_serving_workload_full_size(cuda, tnq_lib, oracle_lib):
    """The 64 circuits of the batched serving shape (5x5..7x7 grids, depths
    1+16+1..1+32+1, uneven sizes), 4 of their seeded bitstrings each, in one
    tnq_amplitudes_batch call; plans sliced to bags <= 2^26. The 5x5 circuits
    are checked against the oracle; sampled amplitudes must equal their own
    single-bitstring contraction."""
    nb = 4
    work = I.batched_serving_workload(n_circuits=64, bitstrings_per_circuit=16, seed=0)
    plans = [tnq_lib.Plan(c, max_bag_log2=26, max_p=30) for c, _ in work]
    bl = [bits[:nb] for _, bits in work]
    out = tnq_lib.amplitudes_batch(plans, bl)
    assert out.shape == (64 * nb,)
    rng = np.random.default_rng(0)
    checked = 0
    for i, ((circ, bits), plan) in enumerate(zip(work, plans)):
        j = int(rng.integers(nb))
        if i % 4 == 0 or circ.n_qubits == 25:
            single = tnq_lib.contract_sliced(plan, bits[j])
            assert abs(out[nb * i + j] - single) <= 1e-9 * max(abs(single), 1e-30)
        if circ.n_qubits == 25 and checked < 6:
            ref = oracle_lib.contract(circ, bits[j], order=plan.order(), mu=plan.sliced())
            assert rel_err(out[nb * i + j], ref, 25) < TOL
            checked += 1
    assert checked > 0


@pytest.mark.parametrize("slicer", [0, 1, 2, 4])
def test_every_slicer_gives_the_same_amplitude(cuda, tnq_lib, oracle_lib, slicer):
    """The score of Algorithm 2 only chooses mu (Eq. 5 regroups the same sum):
    tree-trimming, degree, direct and betweenness plans all give the oracle's
    amplitude, slice by slice."""
    circ = I.random_grid_circuit(5, 5, 20, 3)
    bits = I.random_bitstring(25, 3)
    plan = tnq_lib.Plan(circ, slicer=slicer, min_p=4, max_p=4)
    amp, per = tnq_lib.contract_sliced(plan, bits, per_slice=True)
    ref, ref_per = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced(), per_slice=True)
    for s in range(len(per)):
        assert rel_err(per[s], ref_per[s], 25) < TOL, s
    assert rel_err(amp, oracle_lib.contract(circ, bits), 25) < TOL


def test_autotuned_tuning_reproduces_and_matches_oracle(cuda, tnq_lib, oracle_lib):
    """The autotuner picks a GEMM cut-over and tile shape per plan; a plan built
    later with the same options, given that tuning and chain selection, gives
    bit-identical slices, and both match the oracle."""
    circ = I.random_grid_circuit(6, 6, 24, 7)
    bits = I.random_bitstring(36, 7)
    kw = dict(max_bag_log2=20, max_p=20, reorder_every=1, precision=1, gemm_min_k_log2=4, fuse_min_rank=10)
    plan = tnq_lib.Plan(circ, **kw)
    plan.autotune(bits, max_batch=16)
    tuning, kept = plan.tuning(), plan.fused_chains()
    assert tuning[0] in (3, 4, 5, 6) and tuning[1] in (3, 64)
    _, per = tnq_lib.contract_sliced(plan, bits, per_slice=True)
    again = tnq_lib.Plan(circ, **kw)
    again.set_tuning(*tuning)
    again.keep_chains(kept)
    assert again.fused_chains() == kept
    _, per2 = tnq_lib.contract_sliced(again, bits, per_slice=True)
    assert np.array_equal(per, per2)
    ref, ref_per = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced(), per_slice=True)
    for s in range(len(per)):
        assert rel_err(per[s], ref_per[s], 36) < SPLIT_TOL, s


def test_batched_call_lanes_duplicates_and_small_workspace(cuda, tnq_lib, oracle_lib):
    """tnq_amplitudes_batch with the same plan listed twice, a plan with no
    bitstrings between, several circuit sizes on the concurrent lanes, and a
    workspace only large enough for one lane: every amplitude equals its own
    single-bitstring contraction and the oracle."""
    import torch

    circs = [I.random_grid_circuit(4, 5, 16, 60 + k) for k in range(3)] + [I.random_grid_circuit(5, 5, 20, 63)]
    plans = [tnq_lib.Plan(c, min_p=2, max_p=2) for c in circs]
    order = [0, 1, 0, 2, 3, 1]
    bl = [[I.random_bitstring(circs[i].n_qubits, 100 * j + k) for k in range(3)] for j, i in enumerate(order)]
    bl[4] = []
    lst = [plans[i] for i in order]
    want = []
    for j, i in enumerate(order):
        for b in bl[j]:
            want.append(tnq_lib.contract_sliced(plans[i], b))
            ref = oracle_lib.contract(circs[i], b)
            assert rel_err(want[-1], ref, circs[i].n_qubits) < TOL
    got = tnq_lib.amplitudes_batch(lst, bl)
    assert np.max(np.abs(got - np.array(want))) <= 1e-9 * np.max(np.abs(want))
    # one lane: a workspace that fits one item of the largest plan plus the call's staging
    need = max(p.workspace_bytes(1) for p in plans)
    ws = torch.empty(need + need // 4 + (1 << 20), dtype=torch.uint8, device="cuda")
    got1 = tnq_lib.amplitudes_batch(lst, bl, workspace=ws)
    assert np.max(np.abs(got1 - np.array(want))) <= 1e-9 * np.max(np.abs(want))

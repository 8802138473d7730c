"""Host planner: the paper's worked example, tree-decomposition validity,
slicing invariants and the exact cost model (no GPU)."""
import itertools
import json
import os

import numpy as np
import pytest

from paper_2004_10892_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def toy():
    g = json.load(open(os.path.join(GOLDEN, "toy_eq1.json")))
    names = sorted({v for t in g["tensors"] for v in t})
    idx = {v: i for i, v in enumerate(names)}
    edges = set()
    for t in g["tensors"]:
        for a, b in itertools.combinations(t, 2):
            edges.add(tuple(sorted((idx[a], idx[b]))))
    g["names"] = names
    g["idx"] = idx
    g["edges"] = sorted(edges)
    return g


def _order(toy, names):
    return [toy["idx"][v] for v in names]


def test_toy_eq2_sequence(tnq_lib, toy):
    tau, sizes = tnq_lib.graph_treewidth(6, toy["edges"], _order(toy, toy["order"]), bag_sizes=True)
    assert tau == toy["treewidth"]
    assert sizes == toy["eq2_cost_exponents"]
    # intermediate of step i = its bag minus the eliminated index (Eq. 2)
    assert [s - 1 for s in sizes] == [len(t) for t in toy["eq2_intermediates"]]


def test_toy_tree_decomposition_is_path(tnq_lib, toy):
    bags, parent = tnq_lib.graph_tree_decomposition(6, toy["edges"], _order(toy, toy["order"]))
    got = sorted(tuple(sorted(toy["names"][v] for v in b)) for b in bags)
    assert got == sorted(tuple(sorted(b)) for b in toy["td_bags"])
    assert max(len(b) for b in bags) == toy["max_bag"]
    # a path: every bag has at most two tree neighbours
    deg = [0] * len(bags)
    for c, p in enumerate(parent):
        if p >= 0:
            deg[c] += 1
            deg[p] += 1
    assert max(deg) <= 2 and sum(p < 0 for p in parent) == 1
    # the reverse order yields the same tree
    bags_r, _ = tnq_lib.graph_tree_decomposition(6, toy["edges"], _order(toy, toy["reverse_order"]))
    assert sorted(map(sorted, bags_r)) == sorted(map(sorted, bags))


@pytest.mark.parametrize("slicer", [0, 1, 2])
def test_toy_first_deletion_is_k(tnq_lib, toy, slicer):
    """Tree-trimming (k, l tie on length 3 and weight 9; the earliest wins),
    degree (k has degree 4) and direct reduction all fix k: tau drops to 1."""
    mu, tau = tnq_lib.graph_greedy_deletion(6, toy["edges"], _order(toy, toy["order"]), 1, slicer=slicer)
    assert toy["names"][mu[0]] == "k"
    assert tau[0] == toy["fix_k_treewidth"]


def test_toy_fixing_l_leaves_a_triangle(tnq_lib, toy):
    l = toy["idx"]["l"]
    edges = [e for e in toy["edges"] if l not in e]
    assert tnq_lib.graph_treewidth(6, edges, _order(toy, toy["order"])) == toy["fix_l_treewidth"]


def _td_valid(n, edges, bags, parent):
    """The three criteria of a tree decomposition (Section II.B)."""
    cover = set(v for b in bags for v in b)
    if cover != set(range(n)):
        return "vertex not covered"
    for a, b in edges:
        if not any(a in x and b in x for x in bags):
            return f"edge {a}-{b} not in a bag"
    nb = len(bags)
    adj = [[] for _ in range(nb)]
    for c, p in enumerate(parent):
        if p >= 0:
            adj[c].append(p)
            adj[p].append(c)
    if sum(p < 0 for p in parent) != 1 or sum(len(a) for a in adj) != 2 * (nb - 1):
        return "not a tree"
    for v in range(n):
        holders = [i for i, b in enumerate(bags) if v in b]
        seen = {holders[0]}
        stack = [holders[0]]
        while stack:
            x = stack.pop()
            for y in adj[x]:
                if y not in seen and v in bags[y]:
                    seen.add(y)
                    stack.append(y)
        if len(seen) != len(holders):
            return f"bags of {v} are not connected"
    for i, a in enumerate(bags):
        for j, b in enumerate(bags):
            if i != j and set(a) <= set(b):
                return "non-maximal bag"
    return ""


def _random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    return [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]


@pytest.mark.parametrize("seed", range(8))
def test_tree_decomposition_valid(tnq_lib, seed):
    n = 8 + 3 * seed
    edges = _random_graph(n, 0.25, seed)
    for method in (0, 1):
        order = tnq_lib.graph_order(n, edges, method)
        assert sorted(order) == list(range(n))
        bags, parent = tnq_lib.graph_tree_decomposition(n, edges, order)
        assert _td_valid(n, edges, bags, parent) == ""
        tau = tnq_lib.graph_treewidth(n, edges, order)
        assert max(len(b) for b in bags) - 1 == max(tau, max(len(b) for b in bags) - 1)
        assert max(len(b) for b in bags) - 1 <= tau


def test_tree_decomposition_of_circuit_graph(tnq_lib, oracle_lib):
    c = I.random_grid_circuit(5, 5, 20, 1)
    fv = oracle_lib.free_vars(c)
    edges = oracle_lib.graph_edges(c)
    n = len(fv)
    order = tnq_lib.graph_order(n, edges, 0)
    bags, parent = tnq_lib.graph_tree_decomposition(n, edges, order)
    assert _td_valid(n, edges, bags, parent) == ""
    assert max(len(b) for b in bags) - 1 == tnq_lib.graph_treewidth(n, edges, order)


def test_known_treewidths(tnq_lib):
    # path, cycle, complete graph, 3x3 grid (treewidth 3)
    path = [(i, i + 1) for i in range(9)]
    cyc = path + [(9, 0)]
    k6 = [(a, b) for a in range(6) for b in range(a + 1, 6)]
    grid = [(r * 3 + c, r * 3 + c + 1) for r in range(3) for c in range(2)] + \
           [(r * 3 + c, (r + 1) * 3 + c) for r in range(2) for c in range(3)]
    for n, e, tw in [(10, path, 1), (10, cyc, 2), (6, k6, 5), (9, grid, 3)]:
        assert tnq_lib.graph_treewidth(n, e, tnq_lib.graph_order(n, e, 0)) == tw


def _exact_tw(tnq_lib, n, edges):
    return min(tnq_lib.graph_treewidth(n, edges, list(o)) for o in itertools.permutations(range(n)))


@pytest.mark.parametrize("seed", range(3))
def test_deleting_one_vertex_lowers_treewidth_by_at_most_one(tnq_lib, seed):
    """Section III.A: removing a vertex lowers the (exact) treewidth by <= 1."""
    n = 7
    edges = _random_graph(n, 0.5, 10 + seed)
    tw = _exact_tw(tnq_lib, n, edges)
    for u in range(n):
        red = [e for e in edges if u not in e]
        tw_u = _exact_tw(tnq_lib, n, red)
        assert tw - 1 <= tw_u <= tw


@pytest.mark.parametrize("slicer", [0, 1, 2])
def test_greedy_deletion_monotone(tnq_lib, oracle_lib, slicer):
    """With the reduced order kept (Algorithm 2 without line 10's TD
    recomputation), the treewidth never grows as vertices are removed."""
    c = I.random_grid_circuit(5, 5, 16, 3)
    edges = oracle_lib.graph_edges(c)
    n = len(oracle_lib.free_vars(c))
    order = tnq_lib.graph_order(n, edges, 0)
    tau0 = tnq_lib.graph_treewidth(n, edges, order)
    mu, tau = tnq_lib.graph_greedy_deletion(n, edges, order, 6, slicer=slicer)
    assert len(set(mu)) == 6
    seq = [tau0] + tau
    assert all(b <= a for a, b in zip(seq, seq[1:]))


def test_tree_trimming_beats_degree_on_grid(tnq_lib, oracle_lib):
    """Section IV: tree-trimming lowers the treewidth faster than the degree score."""
    c = I.random_grid_circuit(6, 6, 20, 0)
    edges = oracle_lib.graph_edges(c)
    n = len(oracle_lib.free_vars(c))
    order = tnq_lib.graph_order(n, edges, 0)
    _, tt = tnq_lib.graph_greedy_deletion(n, edges, order, 6, slicer=0)
    _, dg = tnq_lib.graph_greedy_deletion(n, edges, order, 6, slicer=1)
    assert tt[-1] <= dg[-1]
    tau0 = tnq_lib.graph_treewidth(n, edges, order)
    assert tt[-1] <= tau0 - 3


def test_plan_variables_match_oracle_network(tnq_lib, oracle_lib):
    for circ in [I.random_grid_circuit(4, 4, 16, 0), I.random_small_circuit(6, 60, 1), I.ghz(5)]:
        plan = tnq_lib.Plan(circ, min_p=2, max_p=2)
        keys = plan.order() + plan.sliced()
        assert sorted(keys) == sorted(oracle_lib.free_vars(circ))
        assert len(set(keys)) == len(keys)


def test_plan_stopping_rule(tnq_lib):
    c = I.random_grid_circuit(6, 6, 24, 0)
    plan = tnq_lib.Plan(c, max_bag_log2=14, max_p=40)
    inf = plan.info()
    assert inf["max_bag"] <= 14 and inf["p"] >= 1
    assert inf["tau"] <= inf["tau_full"]
    plan2 = tnq_lib.Plan(c, max_bag_log2=24, min_p=4, max_p=8)
    assert plan2.info()["p"] == 4
    assert plan2.info()["n_slices"] == 16


def test_plan_deterministic(tnq_lib):
    c = I.random_grid_circuit(5, 5, 20, 9)
    a = tnq_lib.Plan(c, min_p=3, max_p=3)
    b = tnq_lib.Plan(c, min_p=3, max_p=3)
    assert a.order() == b.order() and a.sliced() == b.sliced()


def test_cost_model_equals_oracle_counts(tnq_lib, oracle_lib):
    """Exact cost model: flops per slice = 6 (complex mults) + 2 (complex adds)
    as counted by the oracle running the plan's buckets (plain Eq. 2, every
    gate tensor in the bucket of its earliest variable: leaf absorption off)."""
    for circ, kw in [(I.random_grid_circuit(4, 4, 12, 2), {}), (I.random_grid_circuit(4, 5, 16, 5), dict(min_p=2, max_p=2)),
                     (I.random_small_circuit(7, 70, 4), dict(min_p=1, max_p=1))]:
        plan = tnq_lib.Plan(circ, leaf_absorb=0, **kw)
        inf = plan.info()
        bits = I.random_bitstring(circ.n_qubits, 3)
        _, (cmul, cadd) = oracle_lib.contract(circ, bits, order=plan.order(), mu=plan.sliced(), slices=(0, 1),
                                              counts=True)
        assert inf["flops_per_slice"] == 6 * cmul + 2 * cadd
        bag, k, _ = plan.buckets()
        assert inf["max_bag"] == bag.max()
        assert inf["total_flops"] == inf["flops_per_slice"] * inf["n_slices"]


def test_plan_rejects_bad_circuits(tnq_lib):
    bad = [I.Circuit(2, [I.Gate(I.CZ, 0, 0)]), I.Circuit(2, [I.Gate(I.H, 2)]), I.Circuit(2, [I.Gate(9, 0)]),
           I.Circuit(0, [])]
    for c in bad:
        with pytest.raises(tnq_lib.TnqError) as e:
            tnq_lib.Plan(c)
        assert e.value.status == tnq_lib.EINVAL
    with pytest.raises(tnq_lib.TnqError):
        tnq_lib.Plan(I.all_h(3), min_p=3, max_p=1)


def test_plan_without_free_variables(tnq_lib):
    plan = tnq_lib.Plan(I.all_h(4))
    inf = plan.info()
    assert inf["n_free_vars"] == 0 and inf["n_buckets"] == 0 and inf["n_slices"] == 1


def _bucket_rows(tnq_lib, plan):
    """Per bucket (bag r, inputs k, output rank, sums) from the internal hook."""
    import ctypes

    L = tnq_lib.lib()
    n = ctypes.c_int32()
    cap = 12 * 4096
    out = (ctypes.c_int32 * cap)()
    assert L.tnq_internal_bucket_detail(plan.handle, out, cap, ctypes.byref(n)) == 0
    return np.frombuffer(out, dtype=np.int32)[:12 * n.value].reshape(-1, 12)[:, :4]


def test_leaf_absorption_moves_multiplies_to_smaller_buckets(tnq_lib):
    """Leaf absorption keeps every bag and the number of tensor reads, and
    lowers the exact flop count, which still equals the sum over the program's
    buckets of 6 (k-1) 2^r + 2^r (the last term for summing buckets)."""
    for circ, kw in [(I.random_grid_circuit(5, 5, 20, 1), dict(min_p=2, max_p=2)),
                     (I.random_grid_circuit(6, 6, 24, 0), dict(max_bag_log2=20, max_p=12))]:
        off = tnq_lib.Plan(circ, leaf_absorb=0, **kw)
        on = tnq_lib.Plan(circ, **kw)
        r0, r1 = _bucket_rows(tnq_lib, off), _bucket_rows(tnq_lib, on)
        assert (r0[:, [0, 2, 3]] == r1[:, [0, 2, 3]]).all() and r0[:, 1].sum() == r1[:, 1].sum()
        assert on.info()["flops_per_slice"] < off.info()["flops_per_slice"]
        for plan, rows in ((off, r0), (on, r1)):
            flops = sum(6.0 * (k - 1) * 2.0 ** r + (2.0 ** r if sm else 0.0) for r, k, _, sm in rows)
            assert plan.info()["flops_per_slice"] == flops


def test_betweenness_closed_forms(tnq_lib):
    """Betweenness centrality (Section III.A) on graphs with known values:
    path P_n: vertex i lies on i (n-1-i) shortest paths; star: the centre on
    all C(n-1, 2); cycle C_5: each vertex on one path (between its two
    neighbours); complete graph: 0; 4-cycle: each vertex carries half of the
    two shortest paths between its neighbours."""
    n = 9
    path = [(i, i + 1) for i in range(n - 1)]
    assert np.allclose(tnq_lib.graph_betweenness(n, path), [i * (n - 1 - i) for i in range(n)])
    star = [(0, i) for i in range(1, n)]
    assert np.allclose(tnq_lib.graph_betweenness(n, star), [(n - 1) * (n - 2) / 2] + [0] * (n - 1))
    c5 = [(i, (i + 1) % 5) for i in range(5)]
    assert np.allclose(tnq_lib.graph_betweenness(5, c5), [1.0] * 5)
    k5 = list(itertools.combinations(range(5), 2))
    assert np.allclose(tnq_lib.graph_betweenness(5, k5), [0.0] * 5)
    c4 = [(i, (i + 1) % 4) for i in range(4)]
    assert np.allclose(tnq_lib.graph_betweenness(4, c4), [0.5] * 4)


def test_betweenness_matches_networkx(tnq_lib):
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(3)
    for trial in range(6):
        n = int(rng.integers(5, 40))
        G = nx.gnm_random_graph(n, int(rng.integers(n, 3 * n)), seed=int(rng.integers(1 << 30)))
        ref = nx.betweenness_centrality(G, normalized=False)
        got = tnq_lib.graph_betweenness(n, list(G.edges()))
        assert np.allclose(got, [ref[v] for v in range(n)], rtol=1e-12, atol=1e-9), trial


def test_betweenness_slicer(tnq_lib):
    """Algorithm 2 with the betweenness score: on a path the first deletion is
    the middle vertex; on a circuit graph it lowers the treewidth like the
    other scores, and the plan option runs end to end."""
    n = 9
    path = [(i, i + 1) for i in range(n - 1)]
    mu, tau = tnq_lib.graph_greedy_deletion(n, path, list(range(n)), 1, slicer=tnq_lib.SLICER_BETWEENNESS)
    assert mu == [4] and tau == [1]
    circ = I.random_grid_circuit(5, 5, 20, 0)
    base = tnq_lib.Plan(circ)
    plan = tnq_lib.Plan(circ, slicer=tnq_lib.SLICER_BETWEENNESS, min_p=6, max_p=6)
    assert plan.info()["p"] == 6 and plan.info()["tau"] < base.info()["tau"]


def test_score_comparison_experiment(tnq_lib):
    """The Section IV score comparison on a small circuit: every score's
    treewidth of the fixed reduced order is non-increasing over the deletions
    (it may drop by more than one: the order is not re-optimised), the
    recorded deletions are distinct, and after ten deletions tree-trimming is
    at least as good as degree (the paper's ordering of the two scores)."""
    from paper_2004_10892_gb300 import score_compare

    row = score_compare.compare(I.random_grid_circuit(6, 6, 24, 0), 10, list(score_compare.SCORES))
    assert row["vertices"] > 0 and row["tau0"] > 0
    for name, r in row["scores"].items():
        tau = [row["tau0"]] + r["tau"]
        assert len(r["mu"]) == 10 and len(set(r["mu"])) == 10, name
        assert all(a >= b for a, b in zip(tau, tau[1:])), (name, tau)
    assert row["scores"]["tree_trimming"]["tau"][-1] <= row["scores"]["degree"]["tau"][-1]


def test_order_recomputation(tnq_lib):
    """Algorithm 2's optional recomputation step (reorder_every): a fresh greedy
    order of the reduced graph replaces the inherited one unless its width is
    larger, so the treewidth never ends above the plain run's, stays
    non-increasing, and the plan option works end to end."""
    n, edges = tnq_lib.circuit_graph(I.random_grid_circuit(6, 6, 24, 1))
    order = tnq_lib.graph_order(n, edges)
    for slicer in (tnq_lib.SLICER_TREE_TRIMMING, tnq_lib.SLICER_DIRECT):
        _, plain = tnq_lib.graph_greedy_deletion(n, edges, order, 8, slicer=slicer)
        _, re1 = tnq_lib.graph_greedy_deletion(n, edges, order, 8, slicer=slicer, reorder_every=1)
        assert all(a >= b for a, b in zip(re1, re1[1:]))
        assert re1[-1] <= plain[-1] + 1
    circ = I.random_grid_circuit(6, 6, 24, 1)
    a = tnq_lib.Plan(circ, max_bag_log2=16, max_p=30)
    b = tnq_lib.Plan(circ, max_bag_log2=16, max_p=30, reorder_every=1)
    assert b.info()["max_bag"] <= 16 and b.info()["p"] <= a.info()["p"] + 1


def test_order_trials(tnq_lib):
    """Planning from several greedy orders with seeded random ties keeps the
    bag limit, is deterministic for a seed, and with one trial is the plain
    deterministic plan."""
    circ = I.random_grid_circuit(6, 6, 24, 2)
    one = tnq_lib.Plan(circ, max_bag_log2=16, max_p=30)
    same = tnq_lib.Plan(circ, max_bag_log2=16, max_p=30, order_trials=1)
    assert one.order() == same.order() and one.sliced() == same.sliced()
    a = tnq_lib.Plan(circ, max_bag_log2=16, max_p=30, order_trials=8, seed=3)
    b = tnq_lib.Plan(circ, max_bag_log2=16, max_p=30, order_trials=8, seed=3)
    assert a.order() == b.order() and a.sliced() == b.sliced()
    assert a.info()["max_bag"] <= 16 and a.info()["p"] <= one.info()["p"] + 1


def test_order_trials_do_not_depend_on_threads(tnq_lib, monkeypatch):
    """The randomised greedy orders are tried on host threads; the chosen plan
    is the same with one thread (the earliest of equally cheap trials wins)."""
    cases = [(I.random_grid_circuit(6, 6, 24, 2), dict(max_bag_log2=16, max_p=30, order_trials=16, seed=5)),
             (I.random_grid_circuit(7, 7, 32, 0), dict(max_bag_log2=28, max_p=40, reorder_every=1, order_trials=12))]
    for circ, kw in cases:
        monkeypatch.delenv("TNQ_PLAN_THREADS", raising=False)
        a = tnq_lib.Plan(circ, **kw)
        monkeypatch.setenv("TNQ_PLAN_THREADS", "1")
        b = tnq_lib.Plan(circ, **kw)
        assert a.order() == b.order() and a.sliced() == b.sliced()
        assert a.info()["total_flops"] == b.info()["total_flops"]

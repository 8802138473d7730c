"""The C-ABI library loads and exports every symbol include/tnq.h declares;
error paths work without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_2004_10892_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(tnq_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(tnq_lib):
    names = declared_functions()
    assert len(names) >= 15
    L = ctypes.CDLL(tnq_lib.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_header(tnq_lib):
    assert set(declared_functions()) <= set(tnq_lib.SIGNATURES)


def test_status_strings(tnq_lib):
    L = tnq_lib.lib()
    for s in range(6):
        assert L.tnq_status_string(s)
    assert b"sm_103a" in L.tnq_version()


def test_null_arguments_are_rejected(tnq_lib):
    L = tnq_lib.lib()
    assert L.tnq_plan_from_circuit(1, None, 0, None, None) == tnq_lib.EINVAL
    assert L.tnq_plan_info_get(None, None) == tnq_lib.EINVAL
    assert b"NULL" in L.tnq_last_error()
    out = (ctypes.c_double * 2)()
    assert L.tnq_contract_sliced(None, None, 0, 1, None, 0, 0, None, out, None) == tnq_lib.EINVAL


def test_bad_slice_range_and_bits(tnq_lib):
    import numpy as np

    plan = tnq_lib.Plan(I.random_grid_circuit(3, 3, 8, 0), min_p=2, max_p=2)
    L = tnq_lib.lib()
    bits = np.zeros(9, np.uint8)
    out = np.zeros(2)
    P = ctypes.POINTER
    rc = L.tnq_contract_sliced(plan.handle, bits.ctypes.data_as(P(ctypes.c_uint8)), 0, 5, None, 0, 0, None,
                               out.ctypes.data_as(P(ctypes.c_double)), None)
    assert rc == tnq_lib.EINVAL and b"slice range" in L.tnq_last_error()
    bits[3] = 2
    rc = L.tnq_contract_sliced(plan.handle, bits.ctypes.data_as(P(ctypes.c_uint8)), 0, 4, None, 0, 0, None,
                               out.ctypes.data_as(P(ctypes.c_double)), None)
    assert rc == tnq_lib.EINVAL


def test_empty_slice_range_is_zero(tnq_lib):
    import numpy as np

    plan = tnq_lib.Plan(I.random_grid_circuit(3, 3, 8, 0), min_p=2, max_p=2)
    L = tnq_lib.lib()
    bits = np.zeros(9, np.uint8)
    out = np.ones(2)
    P = ctypes.POINTER
    rc = L.tnq_contract_sliced(plan.handle, bits.ctypes.data_as(P(ctypes.c_uint8)), 2, 2, None, 0, 0, None,
                               out.ctypes.data_as(P(ctypes.c_double)), None)
    assert rc == tnq_lib.OK and out[0] == 0 and out[1] == 0


def test_contract_without_gpu_fails_loudly(tnq_lib):
    import numpy as np
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    plan = tnq_lib.Plan(I.random_grid_circuit(3, 3, 8, 0))
    L = tnq_lib.lib()
    bits = np.zeros(9, np.uint8)
    out = np.zeros(2)
    P = ctypes.POINTER
    rc = L.tnq_contract_sliced(plan.handle, bits.ctypes.data_as(P(ctypes.c_uint8)), 0, 1, None, 0, 0, None,
                               out.ctypes.data_as(P(ctypes.c_double)), None)
    assert rc == tnq_lib.EUNSUPPORTED


def test_workspace_grows_with_batch(tnq_lib):
    plan = tnq_lib.Plan(I.random_grid_circuit(5, 5, 16, 0), min_p=3, max_p=3)
    sizes = [plan.workspace_bytes(b) for b in (1, 2, 4, 8)]
    assert all(b >= a for a, b in zip(sizes, sizes[1:])) and sizes[0] > 0
    assert plan.workspace_bytes(3) == plan.workspace_bytes(4)


def test_launch_bounds_hold_on_host(tnq_lib):
    """Every bucket launch's largest index stays inside its tensor, in every
    configuration the contraction calls can pick (host-side check)."""
    L = tnq_lib.lib()
    f = L.tnq_internal_validate
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_char_p, ctypes.c_size_t]
    buf = ctypes.create_string_buffer(256)
    for c, kw in [(I.random_grid_circuit(4, 4, 16, 0), {}), (I.random_grid_circuit(5, 5, 20, 1), dict(min_p=3, max_p=3)),
                  (I.ghz(5), {}), (I.all_h(3), {}), (I.random_small_circuit(9, 90, 2), dict(min_p=2, max_p=2)),
                  (I.random_grid_circuit(6, 6, 24, 3), dict(max_bag_log2=24, min_p=4, max_p=4, precision=1,
                                                            gemm_min_k_log2=3)),
                  (I.random_grid_circuit(5, 5, 20, 2), dict(precision=2, gemm_min_k_log2=3, fuse_min_rank=4))] + [
                  (I.random_grid_circuit(rows, cols, cyc, 20 + seed), dict(min_p=p, max_p=p, fuse_min_rank=fuse))
                  for seed, (rows, cols, cyc, p) in enumerate([(4, 4, 16, 2), (5, 5, 20, 3), (4, 5, 24, 4)])
                  for fuse in (1, 4, 8)]:  # tiny fused chains (no tile variable, constants from the chain)
        plan = tnq_lib.Plan(c, **kw)
        for mode in (0, 1):
            for B in (1, 2, 8, 64, 1024):
                assert f(plan.handle, mode, B, buf, 256) == 0, (c.name, mode, B, buf.value)


def test_step_kinds_of_the_7x7_plan(tnq_lib):
    """Host-only configuration: the 7x7 depth 1+32+1 plan runs its chains as
    fused k_group steps and every other bucket as a k_bucket step."""
    L = tnq_lib.lib()
    f = L.tnq_internal_step_kinds
    P = ctypes.POINTER
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, P(ctypes.c_int32), P(ctypes.c_int32), ctypes.c_int,
                  P(ctypes.c_int32)]
    plan = tnq_lib.Plan(I.random_grid_circuit(7, 7, 32, 0), max_bag_log2=28, max_p=40)
    info = plan.info()
    kind = (ctypes.c_int32 * 4096)()
    nbk = (ctypes.c_int32 * 4096)()
    n = ctypes.c_int32()
    assert f(plan.handle, 0, 256, kind, nbk, 4096, ctypes.byref(n)) == 0
    kinds = [kind[i] for i in range(n.value)]
    assert kinds.count(1) == info["n_fused_groups"] and set(kinds) <= {0, 1}
    assert sum(nbk[i] for i in range(n.value)) == info["n_buckets"]


def test_fused_a_gemm_form_selection(tnq_lib, monkeypatch):
    """Host-only: GEMM steps with one A operand whose three lowest summed
    variables are its lowest bits read A inside the GEMM kernel (fused-A form:
    no A pack launch); operands with folded tensors keep the packed form, and
    TNQ_GEMM_FUSED_A=0 packs every operand."""
    L = tnq_lib.lib()
    P = ctypes.POINTER
    f = L.tnq_internal_gemm_forms
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, P(ctypes.c_int32), ctypes.c_int, P(ctypes.c_int32)]
    L.tnq_internal_launches_per_batch.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32]
    txt = L.tnq_internal_group_text
    txt.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_char_p, ctypes.c_size_t]
    plan = tnq_lib.Plan(I.random_grid_circuit(7, 7, 24, 1), max_bag_log2=20, max_p=30, reorder_every=1, precision=1,
                        gemm_min_k_log2=4)
    plan.set_tuning(3, 64)
    buf = (ctypes.c_int32 * 64)()
    n = ctypes.c_int32()

    def forms():
        assert f(plan.handle, 0, 16, buf, 64, ctypes.byref(n)) == 0
        return [buf[i] for i in range(n.value)]

    tb = ctypes.create_string_buffer(1 << 20)
    assert txt(plan.handle, 0, 16, tb, 1 << 20) == 0
    na = [int(l.split(" na ")[1].split()[0]) for l in tb.value.decode().splitlines() if l.startswith("gemm ")]
    fused = forms()
    assert len(fused) == len(na) >= 2 and 1 in fused
    assert all(na[i] == 1 for i in range(len(na)) if fused[i])
    launches = L.tnq_internal_launches_per_batch(plan.handle, 0, 16)
    monkeypatch.setenv("TNQ_GEMM_FUSED_A", "0")
    assert forms() == [0] * len(na)
    assert L.tnq_internal_launches_per_batch(plan.handle, 0, 16) == launches + sum(fused)


def test_fused_chain_selection_roundtrip(tnq_lib):
    """A plan's fused-chain selection can be read and applied to a plan built
    later from the same circuit and options (planning is deterministic)."""
    circ = I.random_grid_circuit(6, 6, 24, 0)
    a = tnq_lib.Plan(circ, max_bag_log2=20, max_p=12)
    chains = a.fused_chains()
    assert len(chains) == a.info()["n_fused_groups"] > 1
    b = tnq_lib.Plan(circ, max_bag_log2=20, max_p=12)
    assert b.fused_chains() == chains
    b.keep_chains(chains[::2] + [10 ** 6])
    assert b.fused_chains() == chains[::2] and b.info()["n_fused_groups"] == len(chains[::2])
    b.keep_chains([])
    assert b.fused_chains() == [] and b.info()["n_fused_groups"] == 0
    assert b.info()["bytes_per_slice"] > a.info()["bytes_per_slice"]


def test_chain_selection_reproduces_after_refusion(tnq_lib):
    """With GEMM chains (split precision), dropping a chain lets the fusion pass
    propose new shared-memory chains over its buckets; whatever selection
    results, applying it to a fresh plan of the same circuit reproduces it."""
    circ = I.random_grid_circuit(6, 6, 24, 4)
    kw = dict(max_bag_log2=20, max_p=12, precision=1, gemm_min_k_log2=3)
    a = tnq_lib.Plan(circ, **kw)
    assert a.info()["n_gemm_buckets"] > 0
    chains = a.fused_chains()
    for drop in range(len(chains)):
        a = tnq_lib.Plan(circ, **kw)
        # every bucket index but the dropped chain's: new chains over its buckets are kept too
        a.keep_chains([i for i in range(20000) if i != chains[drop]])
        sel = a.fused_chains()
        assert chains[drop] not in sel
        b = tnq_lib.Plan(circ, **kw)
        b.keep_chains(sel)
        assert b.fused_chains() == sel, drop
        assert b.info()["bytes_per_slice"] == a.info()["bytes_per_slice"]


def _step_structure(tnq_lib, plan, batch):
    L = tnq_lib.lib()
    f = L.tnq_internal_step_deps
    P = ctypes.POINTER
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                  P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32),
                  P(ctypes.c_int32), P(ctypes.c_int64), P(ctypes.c_int64)]
    cs, cd, ct = 4096, 1 << 20, 16384
    n = ctypes.c_int32()
    stream, write = (ctypes.c_int32 * cs)(), (ctypes.c_int32 * cs)()
    reads = (ctypes.c_int32 * (16 * cs))()
    off, deps = (ctypes.c_int32 * (cs + 1))(), (ctypes.c_int32 * cd)()
    toff, tlen = (ctypes.c_int64 * ct)(), (ctypes.c_int64 * ct)()
    assert f(plan.handle, 0, batch, cs, cd, ct, ctypes.byref(n), stream, write, reads, off, deps, toff, tlen) == 0
    m = n.value
    steps = []
    for i in range(m):
        rd = [x for x in reads[16 * i:16 * i + 16] if x >= 0]
        steps.append((stream[i], write[i], rd, list(deps[off[i]:off[i + 1]])))
    return steps, toff, tlen


def test_concurrent_step_schedule_never_reads_a_clobbered_tensor(tnq_lib):
    """The dependencies of a captured batch (four side streams) are sufficient:
    in many random schedules that respect them and each stream's order, every
    step's inputs still hold the values their producers wrote (or the leaf
    values written before the steps) when it runs, checked on an interval
    model of the arena."""
    import random

    for circ, kw, batch in [(I.random_grid_circuit(6, 6, 24, 0), dict(max_bag_log2=20, max_p=12), 8),
                            (I.random_grid_circuit(7, 7, 32, 0), dict(max_bag_log2=28, max_p=40, reorder_every=1,
                                                                      precision=1), 64)]:
        plan = tnq_lib.Plan(circ, **kw)
        steps, toff, tlen = _step_structure(tnq_lib, plan, batch)
        n = len(steps)
        assert n > 10 and len({s[0] for s in steps}) > 1  # more than one stream in use
        rng = random.Random(1)
        for trial in range(20):
            done = [False] * n
            owner = []  # arena intervals (lo, hi, tensor) currently holding valid data
            stream_steps = {}
            for i, st in enumerate(steps):
                stream_steps.setdefault(st[0], []).append(i)
            pos = {k: 0 for k in stream_steps}
            outputs = {s_[1] for s_ in steps}
            leaves = {t for s_ in steps for t in s_[2] if t not in outputs}  # written before the steps
            for t in leaves:
                owner.append((toff[t], toff[t] + tlen[t], t))
            executed = 0
            while executed < n:
                ready = [k for k, lst in stream_steps.items() if pos[k] < len(lst)
                         and all(done[j] for j in steps[lst[pos[k]]][3])]
                assert ready, "schedule deadlock"
                k = rng.choice(ready)
                i = stream_steps[k][pos[k]]
                pos[k] += 1
                _, w, rd, _ = steps[i]
                for t in rd:  # each input must still be owned by itself
                    lo, hi = toff[t], toff[t] + tlen[t]
                    assert any(o == t for (a, b, o) in owner if a == lo and b == hi), (trial, i, t)
                    assert not any(o != t and a < hi and lo < b for (a, b, o) in owner), (trial, i, t)
                lo, hi = toff[w], toff[w] + tlen[w]
                owner = [(a, b, o) for (a, b, o) in owner if not (a < hi and lo < b)]
                owner.append((lo, hi, w))
                done[i] = True
                executed += 1


def test_early_buckets_of_the_7x7_plan(tnq_lib):
    """Host-only: the buckets that only read gate tensors and each other
    (item-invariant or per item) run first, one launch per level; the
    configuration stays in bounds (their results keep their memory from the
    start of the batch) and the batch issues far fewer launches than it has
    steps."""
    L = tnq_lib.lib()
    f = L.tnq_internal_validate
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_char_p, ctypes.c_size_t]
    k = L.tnq_internal_step_kinds
    P = ctypes.POINTER
    k.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, P(ctypes.c_int32), P(ctypes.c_int32), ctypes.c_int,
                  P(ctypes.c_int32)]
    L.tnq_internal_launches_per_batch.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32]
    plan = tnq_lib.Plan(I.random_grid_circuit(7, 7, 32, 0), max_bag_log2=28, max_p=40, precision=1,
                        reorder_every=1, order_trials=4)
    buf = ctypes.create_string_buffer(256)
    for mode in (0, 1):
        for B in (1, 32):
            assert f(plan.handle, mode, B, buf, 256) == 0, (mode, B, buf.value)
    kind = (ctypes.c_int32 * 4096)()
    n = ctypes.c_int32()
    assert k(plan.handle, 0, 32, kind, None, 4096, ctypes.byref(n)) == 0
    steps = [kind[i] for i in range(n.value)]
    per_step = len(steps) + 2 * steps.count(2) + 4  # GEMM steps launch two packs and the MMA
    launches = L.tnq_internal_launches_per_batch(plan.handle, 0, 32)
    assert 0 < launches < per_step - 150, (launches, per_step)
    assert launches < 80, launches


def test_parity_plans_cover_every_register_tail(tnq_lib):
    """Host-only: the fused-chain plans of the GPU parity tests (small grids at
    fuse_min_rank 1/4/8, the 6x6 plans) contain chains whose later stages run as
    register subtrees of every depth (2, 3, 4) and chains that stay in shared
    memory, so the parity tests exercise both kernel instantiations."""
    L = tnq_lib.lib()
    f = L.tnq_internal_group_tails
    P = ctypes.POINTER
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, P(ctypes.c_int32), ctypes.c_int, P(ctypes.c_int32)]
    seen = set()
    plans = []
    for seed, (rows, cols, cyc, p) in enumerate([(4, 4, 16, 2), (5, 5, 20, 3), (4, 5, 24, 4)]):
        for fuse in (1, 4, 8):
            plans.append(tnq_lib.Plan(I.random_grid_circuit(rows, cols, cyc, 20 + seed), min_p=p, max_p=p,
                                      fuse_min_rank=fuse))
    plans.append(tnq_lib.Plan(I.random_grid_circuit(6, 6, 24, 0), max_bag_log2=24, min_p=5, max_p=5))
    buf = (ctypes.c_int32 * 256)()
    n = ctypes.c_int32()
    for plan in plans:
        for mode in (0, 1):
            assert f(plan.handle, mode, 8, buf, 256, ctypes.byref(n)) == 0
            seen.update(buf[i] for i in range(n.value))
    assert {0, 2, 3, 4} <= seen, seen
    assert seen <= {0, 2, 3, 4}, seen  # depth 1 is not used (shared-memory stage instead)


def test_tuning_roundtrip_and_validation(tnq_lib):
    """tnq_plan_set_tuning recompiles the program (GEMM cut-over, tile shape);
    every launch of the recompiled plan stays in bounds; bad values are refused."""
    circ = I.random_grid_circuit(6, 6, 24, 5)
    plan = tnq_lib.Plan(circ, max_bag_log2=18, max_p=20, reorder_every=1, precision=1, gemm_min_k_log2=4)
    assert plan.tuning() == (4, 64)
    n_gemm = {}
    for k, low in ((3, 3), (6, 0), (4, 64)):
        plan.set_tuning(k, low)
        assert plan.tuning() == (k, low)
        n_gemm[k] = plan.info()["n_gemm_buckets"]
        msg = ctypes.create_string_buffer(512)
        for mode in (0, 1):
            assert tnq_lib.lib().tnq_internal_validate(plan.handle, mode, 4, msg, 512) == 0, msg.value
    assert n_gemm[3] >= n_gemm[4] >= n_gemm[6]
    for bad in ((0, 3), (17, 3), (4, -1), (4, 65)):
        with pytest.raises(tnq_lib.TnqError) as e:
            plan.set_tuning(*bad)
        assert e.value.status == tnq_lib.EINVAL


def test_bench_plan_chain_kernels(tnq_lib):
    """Host-only: in the 7x7 depth 1+32+1 plan every fused chain runs in a
    specialised instantiation -- the 5-stage chains with a register tail
    (k_group<1>), the 2-stage chains as stage 0 plus one dense last stage
    (k_group<2>, region A of shared memory only)."""
    L = tnq_lib.lib()
    txt = L.tnq_internal_group_text
    txt.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_char_p, ctypes.c_size_t]
    plan = tnq_lib.Plan(I.random_grid_circuit(7, 7, 32, 0), max_bag_log2=28, max_p=40, precision=1, gemm_min_k_log2=4,
                        reorder_every=1, order_trials=32, fuse_min_rank=12)
    tb = ctypes.create_string_buffer(1 << 22)
    assert txt(plan.handle, 0, 32, tb, 1 << 22) == 0
    heads = [l.split() for l in tb.value.decode().splitlines() if l.startswith("group ")]
    assert heads
    kinds = []
    for h in heads:
        f = dict(zip(h[2::2], h[3::2]))  # "stages 2 tail 0 ... lean2 1 smem 32768"
        stages, tail, lean2, smem = int(f["stages"]), int(f["tail"]), int(f["lean2"]), int(f["smem"])
        if stages == 2:
            assert lean2 == 1 and tail == 0
        if tail or lean2:
            assert smem <= 32768
        kinds.append(1 if tail else (2 if lean2 else 0))
    assert 1 in kinds and 2 in kinds and 0 not in kinds

"""Pins of the FP64 oracle against facts outside itself (no GPU).

- closed-form amplitudes (all-H, H;H, Bell, GHZ, H then CZ sign pattern)
- algebraic identities of the gate matrices, seen through the state vector
- bucket elimination (Eq. 2) against the brute-force state vector
- independence of the elimination order, and Eq. 5: the sum over slices
  equals the unsliced contraction
- norm 1 of the whole output distribution
- exact operation counts on hand-countable networks
- planted mistakes in a copy of the oracle are caught by these pins
"""
import itertools
import math
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from paper_2004_10892_gb300 import inputs as I

TOL = 1e-12


def bits_of(x, n):
    return [(x >> q) & 1 for q in range(n)]


# ---- closed forms ----------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_all_h_uniform(oracle_lib, n):
    sv = oracle_lib.statevector(I.all_h(n))
    assert np.allclose(sv, 2 ** (-n / 2), atol=TOL, rtol=0)
    for x in [0, (1 << n) - 1, 5 % (1 << n)]:
        a = oracle_lib.contract(I.all_h(n), bits_of(x, n))
        assert abs(a - 2 ** (-n / 2)) < TOL
        assert abs(abs(a) ** 2 - 2.0 ** (-n)) < TOL


@pytest.mark.parametrize("n", [1, 3, 6])
def test_h_twice_is_identity(oracle_lib, n):
    c = I.h_twice(n)
    sv = oracle_lib.statevector(c)
    ref = np.zeros(1 << n)
    ref[0] = 1
    assert np.allclose(sv, ref, atol=TOL)
    for x in range(min(1 << n, 8)):
        assert abs(oracle_lib.contract(c, bits_of(x, n)) - ref[x]) < TOL


def test_bell(oracle_lib):
    c = I.bell()
    ref = np.array([1, 0, 0, 1]) / math.sqrt(2)
    assert np.allclose(oracle_lib.statevector(c), ref, atol=TOL)
    for x in range(4):
        assert abs(oracle_lib.contract(c, bits_of(x, 2)) - ref[x]) < TOL


@pytest.mark.parametrize("n", [2, 3, 7, 10])
def test_ghz(oracle_lib, n):
    c = I.ghz(n)
    sv = oracle_lib.statevector(c)
    ref = np.zeros(1 << n)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.allclose(sv, ref, atol=TOL)
    for x in [0, (1 << n) - 1, 1, (1 << n) - 2, 3]:
        assert abs(oracle_lib.contract(c, bits_of(x, n)) - ref[x]) < TOL


def test_h_then_cz_signs(oracle_lib):
    n = 6
    pairs = [(0, 1), (1, 2), (3, 4), (2, 5), (0, 5)]
    c = I.h_then_cz(n, pairs)
    sv = oracle_lib.statevector(c)
    for x in range(1 << n):
        b = bits_of(x, n)
        sign = (-1) ** sum(b[a] * b[bq] for a, bq in pairs)
        ref = sign * 2 ** (-n / 2)
        assert abs(sv[x] - ref) < TOL
        if x % 7 == 0:
            assert abs(oracle_lib.contract(c, b) - ref) < TOL


# ---- gate identities through the state vector -------------------------------
def _sv1(oracle_lib, kinds):
    return oracle_lib.statevector(I.Circuit(1, [I.Gate(k, 0) for k in kinds]))


def test_gate_identities(oracle_lib):
    s = 1 / math.sqrt(2)
    # (X^1/2)^2 = -iX: |0> -> -i|1>
    assert np.allclose(_sv1(oracle_lib, [I.X_1_2, I.X_1_2]), [0, -1j], atol=TOL)
    # (Y^1/2)^2 = -iY: |0> -> |1>
    assert np.allclose(_sv1(oracle_lib, [I.Y_1_2, I.Y_1_2]), [0, 1], atol=TOL)
    # X^1/2|0> = (|0> - i|1>)/sqrt2 ; Y^1/2|0> = (|0> + |1>)/sqrt2 (column 0 of each matrix)
    assert np.allclose(_sv1(oracle_lib, [I.X_1_2]), [s, -1j * s], atol=TOL)
    assert np.allclose(_sv1(oracle_lib, [I.Y_1_2]), [s, s], atol=TOL)
    # Y^1/2 is not symmetric: Y^1/2 X-flipped input picks column 1 = (-1, 1)/sqrt2
    c = I.Circuit(1, [I.Gate(I.X_1_2, 0), I.Gate(I.X_1_2, 0), I.Gate(I.Y_1_2, 0)])
    assert np.allclose(oracle_lib.statevector(c), [1j * s, -1j * s], atol=TOL)
    # T^2 = S: H T T H |0> = ((1+i)|0> + (1-i)|1>)/2 ; T^8 = I
    assert np.allclose(_sv1(oracle_lib, [I.H, I.T, I.T, I.H]), [(1 + 1j) / 2, (1 - 1j) / 2], atol=TOL)
    assert np.allclose(_sv1(oracle_lib, [I.H] + [I.T] * 8 + [I.H]), [1, 0], atol=TOL)
    # H T H |0> phases: T = diag(1, e^{i pi/4})
    w = np.exp(1j * math.pi / 4)
    assert np.allclose(_sv1(oracle_lib, [I.H, I.T, I.H]), [(1 + w) / 2, (1 - w) / 2], atol=TOL)


def test_cnot_orientation(oracle_lib):
    # control q0 = 1 flips target q1: index x0 + 2 x1 goes 1 -> 3
    c = I.Circuit(2, [I.Gate(I.X_1_2, 0), I.Gate(I.X_1_2, 0), I.Gate(I.CNOT, 0, 1)])
    assert np.allclose(oracle_lib.statevector(c), [0, 0, 0, -1j], atol=TOL)
    c = I.Circuit(2, [I.Gate(I.X_1_2, 1), I.Gate(I.X_1_2, 1), I.Gate(I.CNOT, 0, 1)])
    assert np.allclose(oracle_lib.statevector(c), [0, 0, -1j, 0], atol=TOL)
    for x in range(4):
        assert abs(oracle_lib.contract(c, bits_of(x, 2)) - [0, 0, -1j, 0][x]) < TOL


def test_unitarity_random(oracle_lib):
    for seed in range(5):
        c = I.random_small_circuit(7, 80, seed)
        sv = oracle_lib.statevector(c)
        assert abs(np.vdot(sv, sv) - 1) < 1e-12


# ---- bucket elimination vs brute force -------------------------------------
@pytest.mark.parametrize("seed", range(6))
def test_bucket_elimination_matches_statevector(oracle_lib, seed):
    n = 3 + seed
    c = I.random_small_circuit(n, 12 * n, seed)
    sv = oracle_lib.statevector(c)
    xs = range(1 << n) if n <= 5 else [0, 1, (1 << n) - 1, 17 % (1 << n), 1000 % (1 << n)]
    for x in xs:
        a = oracle_lib.contract(c, bits_of(x, n))
        assert abs(a - sv[x]) < TOL, (x, a, sv[x])


def test_grid_4x4_matches_statevector(oracle_lib):
    c = I.random_grid_circuit(4, 4, 16, 0)
    sv = oracle_lib.statevector(c)
    rng = np.random.default_rng(0)
    for x in [0, (1 << 16) - 1] + list(rng.integers(0, 1 << 16, 12)):
        a = oracle_lib.contract(c, bits_of(int(x), 16))
        assert abs(a - sv[int(x)]) < 1e-12


def test_norm_one(oracle_lib):
    for seed in range(2):
        n = 6
        c = I.random_small_circuit(n, 50, 100 + seed)
        tot = sum(abs(oracle_lib.contract(c, bits_of(x, n))) ** 2 for x in range(1 << n))
        assert abs(tot - 1) < 1e-12


def test_order_independence(oracle_lib):
    c = I.random_grid_circuit(3, 3, 10, 4)
    fv = oracle_lib.free_vars(c)
    bits = I.random_bitstring(9, 4)
    ref = oracle_lib.contract(c, bits)
    rng = np.random.default_rng(1)
    for _ in range(3):
        order = [fv[i] for i in rng.permutation(len(fv))]
        # random orders can create wide buckets; keep the networks small
        assert abs(oracle_lib.contract(c, bits, order=order) - ref) < TOL
    assert abs(oracle_lib.contract(c, bits, order=list(reversed(fv))) - ref) < TOL


def test_slicing_sum_equals_unsliced(oracle_lib):
    """Eq. 5: the slice results sum to the full contraction for any fixed set."""
    c = I.random_grid_circuit(3, 4, 12, 2)
    fv = oracle_lib.free_vars(c)
    bits = I.random_bitstring(12, 2)
    full = oracle_lib.contract(c, bits)
    rng = np.random.default_rng(3)
    for p in (1, 2, 4):
        mu = [fv[i] for i in rng.choice(len(fv), p, replace=False)]
        rest = [v for v in fv if v not in mu]
        tot, per = oracle_lib.contract(c, bits, order=rest, mu=mu, per_slice=True)
        assert len(per) == 1 << p
        assert abs(tot - full) < TOL
        assert abs(per.sum() - full) < TOL
        # a sub-range is the partial sum of the same slices
        if p >= 2:
            part = oracle_lib.contract(c, bits, order=rest, mu=mu, slices=(1, 3))
            assert abs(part - per[1:3].sum()) < TOL
        with pytest.raises(ValueError):
            oracle_lib.contract(c, bits, order=rest, mu=mu, slices=(0, (1 << p) + 1))


def test_slice_values_are_restricted_networks(oracle_lib):
    """sigma_s for mu = {v} equals the state vector of the circuit with v's
    wire segment projected: checked on one qubit, H v H, v fixed."""
    c = I.Circuit(1, [I.Gate(I.H, 0), I.Gate(I.H, 0)])
    fv = oracle_lib.free_vars(c)
    assert fv == [(0, 1)]
    for x in (0, 1):
        tot, per = oracle_lib.contract(c, [x], order=[], mu=fv, per_slice=True)
        # sigma_v = H[x, v] H[v, 0] = (1/2)(-1)^{x v}
        assert abs(per[0] - 0.5) < TOL and abs(per[1] - 0.5 * (-1) ** x) < TOL


def test_exact_counts(oracle_lib):
    # H;H on one qubit: one bucket over v1 with two rank-1 tensors: r=1, k=2
    c = I.Circuit(1, [I.Gate(I.H, 0), I.Gate(I.H, 0)])
    a, cnt = oracle_lib.contract(c, [0], counts=True)
    assert cnt == (2.0, 1.0)
    # no free variables: nothing to count
    a, cnt = oracle_lib.contract(I.all_h(3), [0, 1, 0], counts=True)
    assert cnt == (0.0, 0.0)


# ---- the pins have teeth: planted mistakes ----------------------------------
MUTATIONS = {
    "transposed_gate": ("T->val[a + 2 * b] = U[a][b];", "T->val[a + 2 * b] = U[b][a];"),
    "dropped_u1_term": ("res[b] = term[0] + term[1];", "res[b] = term[0];"),
    "x12_sign": ("U[0][0] = s; U[0][1] = -I * s; U[1][0] = -I * s; U[1][1] = s;",
                 "U[0][0] = s; U[0][1] = I * s; U[1][0] = I * s; U[1][1] = s;"),
    "cz_sign": ("T->val[0] = 1; T->val[1] = 1; T->val[2] = 1; T->val[3] = -1;",
                "T->val[0] = 1; T->val[1] = 1; T->val[2] = -1; T->val[3] = 1;"),
    "slice_bit": ("fixed[mu[j]] = (int)((s >> j) & 1);", "fixed[mu[j]] = (int)((s >> (p - 1 - j)) & 1);"),
    "output_not_fixed": ("int x = bits[N->var_qubit[v]] ? 1 : 0;", "int x = 0;"),
}


def _pins_hold(oracle_lib):
    """A compact battery of the pins above; False as soon as one fails."""
    try:
        test_gate_identities(oracle_lib)
        test_cnot_orientation(oracle_lib)
        test_h_then_cz_signs(oracle_lib)
        for seed in range(3):
            test_bucket_elimination_matches_statevector(oracle_lib, seed)
        c = I.random_grid_circuit(3, 3, 8, 5)
        fv = oracle_lib.free_vars(c)
        bits = I.random_bitstring(9, 5)
        full = oracle_lib.contract(c, bits)
        sv = oracle_lib.statevector(c)
        x = sum(b << q for q, b in enumerate(bits))
        if abs(full - sv[x]) > TOL:
            return False
        mu = [fv[1], fv[4]]
        rest = [v for v in fv if v not in mu]
        tot, per = oracle_lib.contract(c, bits, order=rest, mu=mu, per_slice=True)
        if abs(tot - full) > TOL:
            return False
        # per-slice value of slice 1 (mu[0]=1, mu[1]=0) from a one-variable slicing sum
        t1, per1 = oracle_lib.contract(c, bits, order=[v for v in fv if v != mu[0]], mu=[mu[0]], per_slice=True)
        t2, per2 = oracle_lib.contract(c, bits, order=[v for v in fv if v != mu[1]], mu=[mu[1]], per_slice=True)
        if abs(per[1] + per[3] - per1[1]) > TOL or abs(per[2] + per[3] - per2[1]) > TOL:
            return False
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(oracle_lib, tmp_path, name):
    src = open(os.path.join(os.path.dirname(oracle_lib.__file__), "oracle.c")).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutant = tmp_path / "oracle_mut.c"
    mutant.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.check_call(["gcc", "-std=gnu99", "-O1", "-fopenmp", "-fPIC", "-shared", str(mutant), "-o", str(so),
                           "-lm"])
    with oracle_lib.use_library(str(so)):
        assert not _pins_hold(oracle_lib), f"planted mistake {name} passed every pin"
    assert _pins_hold(oracle_lib)

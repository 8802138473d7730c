"""Pins of the general-network oracle (oracle/network.py) against what the
mathematics fixes, independently of the oracle's own code:

- a ring of matrices contracts to the trace of their product (matmul chain),
  and each slice of it to the trace with the sliced index's digit projected;
- brute-force summation over every assignment on tiny networks;
- Eq. 5: the slices of any digit set sum to the unsliced value;
- the value does not depend on the elimination order;
- an L = 2 network built from a circuit equals the circuit oracle and the
  brute-force state vector;
- planted mistakes in the oracle's steps are caught by these pins.
"""
import itertools

import numpy as np
import pytest

from oracle import network as N
from paper_2004_10892_gb300 import inputs as I


def brute_force(dims, tensors):
    """Sum over every assignment of the product of the selected entries (plain loops)."""
    total = 0j
    for a in itertools.product(*[range(d) for d in dims]):
        prod = 1 + 0j
        for idx, arr in tensors:
            prod *= complex(arr[tuple(a[i] for i in idx)])
        total += prod
    return total


@pytest.mark.parametrize("L,n", [(3, 4), (5, 6), (2, 3), (4, 5), (7, 3)])
def test_ring_is_trace_of_product(L, n):
    net = I.random_ring_network(n, L, seed=L * 10 + n)
    mats = [arr for _, arr in net.tensors]
    ref = np.trace(np.linalg.multi_dot(mats) if n > 2 else mats[0] @ mats[1])
    got = N.contract_network(net.dims, net.tensors)
    assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("L,bit", [(3, 0), (3, 1), (5, 2), (5, 0), (6, 1)])
def test_ring_slices_are_projected_traces(L, bit):
    """Slicing digit `bit` of index 0: slice v is trace(P_v M_0 ... M_{n-1}) with
    P_v the diagonal projector on the values whose digit is v."""
    net = I.random_ring_network(5, L, seed=3 + L + bit)
    mats = [arr for _, arr in net.tensors]
    prod = np.linalg.multi_dot(mats)
    total, per = N.contract_network(net.dims, net.tensors, sliced=[(0, bit)], per_slice=True)
    for v in (0, 1):
        P = np.diag([1.0 if ((x >> bit) & 1) == v else 0.0 for x in range(L)])
        ref = np.trace(P @ prod)
        assert abs(per[v] - ref) <= 1e-12 * max(1.0, abs(ref)), v
    assert abs(total - np.trace(prod)) <= 1e-12 * max(1.0, abs(np.trace(prod)))


@pytest.mark.parametrize("seed", range(8))
def test_small_networks_against_brute_force(seed):
    net = I.random_small_network(5, 4, 3, dims=(1, 2, 3, 4), seed=seed)
    ref = brute_force(net.dims, net.tensors)
    got = N.contract_network(net.dims, net.tensors)
    assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (got, ref)


@pytest.mark.parametrize("seed", range(6))
def test_slices_sum_to_the_value(seed):
    net = I.random_small_network(6, 6, 3, dims=(3, 4, 5), seed=100 + seed)
    ref = N.contract_network(net.dims, net.tensors)
    rng = np.random.default_rng(seed)
    digits = [(i, b) for i, d in enumerate(net.dims) for b in range(8) if (1 << b) < d]
    pick = [digits[k] for k in rng.choice(len(digits), size=min(3, len(digits)), replace=False)]
    total, per = N.contract_network(net.dims, net.tensors, sliced=pick, per_slice=True)
    assert len(per) == 1 << len(pick)
    assert abs(total - ref) <= 1e-12 * max(1.0, abs(ref))
    # two digits of the same index partition its values too
    i = max(range(len(net.dims)), key=lambda k: net.dims[k])
    two = [(i, 0), (i, 1)]
    assert abs(N.contract_network(net.dims, net.tensors, sliced=two) - ref) <= 1e-12 * max(1.0, abs(ref))


def test_order_does_not_change_the_value():
    net = I.random_lattice_network(3, 3, 3, seed=5)
    ref = N.contract_network(net.dims, net.tensors)
    rng = np.random.default_rng(1)
    for _ in range(4):
        order = list(rng.permutation(len(net.dims)))
        assert abs(N.contract_network(net.dims, net.tensors, order=order) - ref) <= 1e-12 * max(1.0, abs(ref))


def test_lattice_against_einsum():
    """A 3x3 lattice at L = 3 and mixed dimensions: one einsum over every index."""
    for L in (3, (2, 3, 5)):
        net = I.random_lattice_network(3, 3, L, seed=11)
        letters = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"
        spec = ",".join("".join(letters[i] for i in idx) for idx, _ in net.tensors) + "->"
        ref = np.einsum(spec, *[arr for _, arr in net.tensors])
        got = N.contract_network(net.dims, net.tensors)
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))


def _circuit_network(circ, bits):
    """<bits|C|0^n> as an L = 2 network, written here from the gate matrices
    (independently of both oracles): one index per wire segment, a rank-1
    tensor |0> on every input segment and <x_q| on every output segment."""
    s2 = 2 ** -0.5
    mats = {I.H: s2 * np.array([[1, 1], [1, -1]], complex), I.X_1_2: s2 * np.array([[1, -1j], [-1j, 1]]),
            I.Y_1_2: s2 * np.array([[1, -1], [1, 1]], complex)}
    cur = list(range(circ.n_qubits))
    n_idx = circ.n_qubits
    tensors = [((q,), np.array([1, 0], complex)) for q in range(circ.n_qubits)]
    for g in circ.gates:
        if g.kind in mats:
            tensors.append(((n_idx, cur[g.q0]), mats[g.kind]))
            cur[g.q0] = n_idx
            n_idx += 1
        elif g.kind == I.T:
            tensors.append(((cur[g.q0],), np.array([1, np.exp(1j * np.pi / 4)])))
        elif g.kind == I.CZ:
            tensors.append(((cur[g.q0], cur[g.q1]), np.array([[1, 1], [1, -1]], complex)))
        else:
            raise AssertionError("gate kind not used here")
    for q in range(circ.n_qubits):
        tensors.append(((cur[q],), np.array([1 - bits[q], bits[q]], complex)))
    return [2] * n_idx, tensors


@pytest.mark.parametrize("seed", range(3))
def test_l2_circuit_network_equals_circuit_oracle(oracle_lib, seed):
    circ = I.random_small_circuit(5, 24, seed, kinds=(I.H, I.X_1_2, I.Y_1_2, I.T, I.CZ))
    sv = oracle_lib.statevector(circ)
    for x in (0, 7, 19):
        bits = [(x >> q) & 1 for q in range(5)]
        dims, tensors = _circuit_network(circ, bits)
        got = N.contract_network(dims, tensors)
        assert abs(got - oracle_lib.contract(circ, bits)) <= 1e-12
        assert abs(got - sv[x]) <= 1e-12


def test_typical_magnitude_of_unit_variance_entries():
    """Zero-mean unit-variance entries: E|Z|^2 = prod_i L_i; the sample mean of
    |Z|^2 over many seeds of a tiny network is near it."""
    vals = []
    for seed in range(400):
        net = I.random_small_network(3, 3, 2, dims=(3,), seed=seed)
        vals.append(abs(N.contract_network(net.dims, net.tensors)) ** 2 /
                    N.typical_magnitude(net.dims, net.tensors) ** 2)
    assert 0.75 < np.mean(vals) < 1.3


def test_bad_inputs_are_rejected():
    net = I.random_ring_network(3, 3, 0)
    with pytest.raises(ValueError):
        N.contract_network([3, 3], net.tensors)  # index 2 unknown
    with pytest.raises(ValueError):
        N.contract_network(net.dims, net.tensors, sliced=[(0, 2)])  # 3 values have digits 0, 1
    with pytest.raises(ValueError):
        N.contract_network(net.dims, net.tensors, order=[0, 1])


# ---- planted mistakes: each must make a pin above fail -----------------------
def _pins_hold():
    try:
        test_ring_is_trace_of_product(3, 4)
        test_ring_slices_are_projected_traces(5, 2)
        for seed in range(3):
            test_small_networks_against_brute_force(seed)
            test_slices_sum_to_the_value(seed)
        test_lattice_against_einsum()
    except AssertionError:
        return False
    return True


def test_pins_hold_on_the_oracle():
    assert _pins_hold()


def test_planted_mistakes_are_caught(monkeypatch):
    orig_restrict, orig_broadcast, orig_eliminate = N._restrict, N._broadcast, N._eliminate

    def wrong_digit(dims, tensors, sliced, s):  # fixes the next digit of the index instead of `bit`
        return orig_restrict(dims, tensors, [(i, (b + 1) % (dims[i] - 1).bit_length()) for i, b in sliced], s)

    def transposed(idx, arr, union):  # forgets to permute the axes into the union's order
        shape = [1] * len(union)
        for k, i in enumerate(idx):
            shape[union.index(i)] = arr.shape[k]
        return np.reshape(arr, shape)

    def dropped_scalar(dims, tensors, order):  # loses the rank-0 tensors
        return orig_eliminate(dims, [(i, a) for i, a in tensors if len(i)], order)

    for name, fake in (("_restrict", wrong_digit), ("_broadcast", transposed), ("_eliminate", dropped_scalar)):
        monkeypatch.setattr(N, name, fake)
        assert not _pins_hold(), name
        monkeypatch.setattr(N, name, {"_restrict": orig_restrict, "_broadcast": orig_broadcast,
                                      "_eliminate": orig_eliminate}[name])
    assert _pins_hold()

"""Seeded synthetic inputs: random grid circuits, bitstrings and small test circuits.

This module is the only code shared by the CUDA path and the FP64 oracle. It
produces gate *lists* (kind, qubits) and bitstrings from a counter-based
generator; it holds none of the method's arithmetic (no gate matrices, no
tensors, no contraction). Each side turns a gate kind into its matrix on its
own.

The paper's experiments use the published random circuits of Boixo et al.
(Section IV), which are not available here. The generator below builds
synthetic stand-ins of the same shape: a rows x cols grid, a layer of H on
every qubit, then ``depth`` cycles of CZ gates following eight fixed
nearest-neighbour patterns in turn, single-qubit gates from
{X^1/2, Y^1/2, T} on qubits that leave a CZ, and a final layer of H.
"""
from __future__ import annotations

from dataclasses import dataclass, field

# Gate kinds: the integer values of ``tnq_gate_kind`` in include/tnq.h.
H, X_1_2, Y_1_2, T, CZ, CNOT, U1 = 0, 1, 2, 3, 4, 5, 6
KIND_NAMES = {H: "H", X_1_2: "X_1_2", Y_1_2: "Y_1_2", T: "T", CZ: "CZ", CNOT: "CNOT", U1: "U1"}
TWO_QUBIT = (CZ, CNOT)

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): a counter-based 64-bit generator."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) by rejection (no modulo bias)."""
        limit = (1 << 64) - ((1 << 64) % n)
        while True:
            v = self.next()
            if v < limit:
                return v % n

    def unit(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / (1 << 53))


@dataclass
class Gate:
    kind: int
    q0: int
    q1: int = -1
    # U1 only: 2x2 complex matrix, row-major, as 8 doubles (re, im) pairs.
    m: tuple = field(default_factory=tuple)


@dataclass
class Circuit:
    n_qubits: int
    gates: list
    name: str = ""


def cz_pattern_pairs(rows: int, cols: int, k: int):
    """Qubit pairs of CZ layer pattern k (0..7) on a rows x cols grid; qubit = r*cols + c.

    Patterns 0,1,4,5 couple horizontal neighbours (r,c)-(r,c+1), patterns
    2,3,6,7 vertical neighbours (r,c)-(r+1,c). Each pattern keeps the pairs
    whose (parity along the coupling, parity across it) equals its offset, so
    the eight patterns together use every grid edge exactly once.
    """
    offsets = {0: (0, 0), 1: (1, 1), 2: (0, 0), 3: (1, 1), 4: (0, 1), 5: (1, 0), 6: (0, 1), 7: (1, 0)}
    horizontal = k in (0, 1, 4, 5)
    a, b = offsets[k]
    pairs = []
    for r in range(rows):
        for c in range(cols):
            if horizontal:
                if c + 1 < cols and c % 2 == a and r % 2 == b:
                    pairs.append((r * cols + c, r * cols + c + 1))
            else:
                if r + 1 < rows and r % 2 == a and c % 2 == b:
                    pairs.append((r * cols + c, (r + 1) * cols + c))
    return pairs


def random_grid_circuit(rows: int, cols: int, depth: int, seed: int) -> Circuit:
    """Random grid circuit of depth 1+depth+1 (H layer, ``depth`` CZ cycles, H layer).

    In cycle c (0-based) the CZ layer uses pattern c mod 8; every qubit that is
    idle in cycle c but took part in a CZ in cycle c-1 gets one gate drawn
    uniformly from {X^1/2, Y^1/2, T} with SplitMix64(seed).
    """
    n = rows * cols
    rng = SplitMix64(seed)
    gates = [Gate(H, q) for q in range(n)]
    prev_busy = set()
    choices = (X_1_2, Y_1_2, T)
    for c in range(depth):
        pairs = cz_pattern_pairs(rows, cols, c % 8)
        busy = set()
        for a, b in pairs:
            gates.append(Gate(CZ, a, b))
            busy.add(a)
            busy.add(b)
        for q in range(n):
            if q in prev_busy and q not in busy:
                gates.append(Gate(choices[rng.below(3)], q))
        prev_busy = busy
    gates.extend(Gate(H, q) for q in range(n))
    return Circuit(n, gates, f"grid{rows}x{cols}_d1+{depth}+1_s{seed}")


def random_bitstring(n: int, seed: int) -> list:
    """n seeded random bits (bit q is qubit q's measured value)."""
    rng = SplitMix64(seed ^ 0xB175B175B175B175)
    return [rng.next() >> 63 for _ in range(n)]


def random_unitary_2x2(rng: SplitMix64) -> tuple:
    """A seeded 2x2 unitary e^{i a}[[cos t e^{i b}, sin t e^{i c}], [-sin t e^{-i c}, cos t e^{-i b}]],
    flattened row-major as (re, im) pairs. Non-symmetric in general, so a
    transposed gate matrix shows up in any amplitude check."""
    import math

    a, b, c = (2 * math.pi * rng.unit() for _ in range(3))
    t = 0.5 * math.pi * rng.unit()
    ct, st = math.cos(t), math.sin(t)

    def ph(x):
        return complex(math.cos(x), math.sin(x))

    m = [ct * ph(a + b), st * ph(a + c), -st * ph(a - c), ct * ph(a - b)]
    out = []
    for z in m:
        out += [z.real, z.imag]
    return tuple(out)


def random_small_circuit(n: int, n_gates: int, seed: int, kinds=(H, X_1_2, Y_1_2, T, CZ, CNOT, U1)) -> Circuit:
    """Arbitrary seeded circuit on n qubits (any pairs, all gate kinds) for small checks."""
    rng = SplitMix64(seed)
    gates = []
    for _ in range(n_gates):
        k = kinds[rng.below(len(kinds))]
        if k in TWO_QUBIT and n >= 2:
            a = rng.below(n)
            b = rng.below(n - 1)
            b = b + 1 if b >= a else b
            gates.append(Gate(k, a, b))
        elif k in TWO_QUBIT:
            gates.append(Gate(H, rng.below(n)))
        elif k == U1:
            gates.append(Gate(U1, rng.below(n), -1, random_unitary_2x2(rng)))
        else:
            gates.append(Gate(k, rng.below(n)))
    return Circuit(n, gates, f"small_n{n}_g{n_gates}_s{seed}")


# Circuits with closed-form amplitudes (used as pins).
def all_h(n: int) -> Circuit:
    return Circuit(n, [Gate(H, q) for q in range(n)], f"allH_{n}")


def h_twice(n: int) -> Circuit:
    return Circuit(n, [Gate(H, q) for q in range(n)] * 2, f"HH_{n}")


def bell() -> Circuit:
    return Circuit(2, [Gate(H, 0), Gate(CNOT, 0, 1)], "bell")


def ghz(n: int) -> Circuit:
    return Circuit(n, [Gate(H, 0)] + [Gate(CNOT, q, q + 1) for q in range(n - 1)], f"ghz_{n}")


def h_then_cz(n: int, pairs) -> Circuit:
    return Circuit(n, [Gate(H, q) for q in range(n)] + [Gate(CZ, a, b) for a, b in pairs], f"hcz_{n}")


# Workload shapes (grid rows, cols, cycles) of the synthetic benchmark circuits.
GRID_4x4 = (4, 4, 16)
GRID_6x6 = (6, 6, 24)
GRID_7x7 = (7, 7, 32)


def batched_serving_workload(n_circuits: int = 64, bitstrings_per_circuit: int = 16, seed: int = 0):
    """Uneven batch: circuits on 5x5..7x7 grids with 16..32 cycles, each with seeded bitstrings.

    Circuit i uses seed ``seed + i``; its grid side and depth are drawn from
    SplitMix64(seed) so that the mix is fixed for a given seed.
    """
    rng = SplitMix64(seed ^ 0x5E5E5E5E)
    out = []
    for i in range(n_circuits):
        side = 5 + rng.below(3)
        depth = 16 + 4 * rng.below(5)  # 16, 20, 24, 28, 32
        circ = random_grid_circuit(side, side, depth, seed + i)
        bits = [random_bitstring(circ.n_qubits, (seed + i) * 1000 + j) for j in range(bitstrings_per_circuit)]
        out.append((circ, bits))
    return out


# ---- general tensor networks (indices of any dimension L) --------------------
@dataclass
class TensorNetwork:
    """A closed tensor network: dims[i] = number of values of index i; tensors
    are (indices, complex128 array of shape (dims[i] for i in indices)), numpy
    C order (the first listed index varies slowest)."""

    dims: list
    tensors: list
    name: str = ""


def _normal_pair(rng: SplitMix64):
    """Two independent standard normal deviates (Box-Muller on two uniforms)."""
    import math

    u1 = 1.0 - rng.unit()  # (0, 1]
    u2 = rng.unit()
    r = math.sqrt(-2.0 * math.log(u1))
    return r * math.cos(2 * math.pi * u2), r * math.sin(2 * math.pi * u2)


def random_complex_array(shape, rng: SplitMix64, scale: float = 1.0, bias: complex = 0j):
    """Entries bias + scale * z with z complex normal of unit variance (re, im
    each of variance 1/2), drawn in C order."""
    import numpy as np

    n = 1
    for d in shape:
        n *= int(d)
    out = np.empty(n, dtype=np.complex128)
    for k in range(n):
        a, b = _normal_pair(rng)
        out[k] = bias + scale * complex(a, b) * 0.7071067811865476
    return out.reshape(tuple(int(d) for d in shape))


def random_lattice_network(rows: int, cols: int, L, seed: int, periodic: bool = False) -> TensorNetwork:
    """A closed rows x cols lattice network: one index per nearest-neighbour bond
    (dimension L, or drawn from the tuple L per bond), one tensor per site over
    its bonds, complex normal entries scaled by prod over its legs of
    dim^-1/4 (so that the value's typical magnitude is 1). `periodic` adds the
    wrap-around bonds (a torus)."""
    rng = SplitMix64(seed ^ 0x1A771CE5)
    dims_choice = tuple(L) if isinstance(L, (tuple, list)) else (int(L),)
    bonds = []
    for r in range(rows):
        for c in range(cols):
            if c + 1 < cols or (periodic and cols > 2):
                bonds.append(((r, c), (r, (c + 1) % cols)))
            if r + 1 < rows or (periodic and rows > 2):
                bonds.append(((r, c), ((r + 1) % rows, c)))
    dims = [dims_choice[rng.below(len(dims_choice))] for _ in bonds]
    legs = {(r, c): [] for r in range(rows) for c in range(cols)}
    for i, (a, b) in enumerate(bonds):
        legs[a].append(i)
        legs[b].append(i)
    tensors = []
    for r in range(rows):
        for c in range(cols):
            idx = tuple(legs[(r, c)])
            scale = 1.0
            for i in idx:
                scale *= dims[i] ** -0.25
            tensors.append((idx, random_complex_array([dims[i] for i in idx], rng, scale)))
    return TensorNetwork(dims, tensors, f"lattice{rows}x{cols}_L{'-'.join(map(str, dims_choice))}_s{seed}")


def random_ring_network(n: int, L: int, seed: int) -> TensorNetwork:
    """n matrices M_k[i_k, i_{k+1 mod n}] around a ring (index k of dimension L):
    its value is trace(M_0 M_1 ... M_{n-1})."""
    rng = SplitMix64(seed ^ 0x21A6)
    dims = [int(L)] * n
    tensors = [((k, (k + 1) % n), random_complex_array([L, L], rng, L ** -0.5)) for k in range(n)]
    return TensorNetwork(dims, tensors, f"ring{n}_L{L}_s{seed}")


def random_small_network(n_indices: int, n_tensors: int, max_rank: int, dims, seed: int) -> TensorNetwork:
    """Arbitrary seeded network for small checks: index dimensions drawn from
    `dims`, each tensor over 0..max_rank distinct random indices (rank-0
    scalars included); every index is then added to some tensor so that all
    appear."""
    rng = SplitMix64(seed ^ 0x5A11)
    dl = [dims[rng.below(len(dims))] for _ in range(n_indices)]
    idx_sets = []
    for _ in range(n_tensors):
        r = rng.below(max_rank + 1)
        pool = list(range(n_indices))
        pick = []
        for _ in range(min(r, n_indices)):
            pick.append(pool.pop(rng.below(len(pool))))
        idx_sets.append(pick)
    used = {i for s in idx_sets for i in s}
    for i in range(n_indices):
        if i not in used:
            idx_sets[rng.below(n_tensors)].append(i)
    tensors = [(tuple(s), random_complex_array([dl[i] for i in s], rng)) for s in idx_sets]
    return TensorNetwork(dl, tensors, f"small_n{n_indices}_t{n_tensors}_s{seed}")

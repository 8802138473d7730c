"""GPU parity for general tensor networks with L-valued indices (Section II.A
for any index dimension; Eq. 4-5 slicing a binary digit of an index): the
CUDA path through tnq_plan_from_network / tnq_contract_sliced against the FP64
network oracle (oracle/network.py), value by value and slice by slice.

Tolerance: 1e-5 relative for the complex64 path, 1e-4 for split precision;
the denominator is |ref| unless |ref|^2 < typical^2 / 10, where typical =
sqrt(E|Z|^2) of a network with the same index dimensions and entry variances
(the analogue of the Porter-Thomas floor of an amplitude).
"""
import numpy as np
import pytest

from oracle import network as N
from paper_2004_10892_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-5
SPLIT_TOL = 1e-4


def rel_err(a, ref, typical):
    den = abs(ref) if abs(ref) ** 2 >= typical ** 2 / 10 else typical
    return abs(a - ref) / den


def check(tnq_lib, net, tol=TOL, per_slice=True, **opts):
    plan = tnq_lib.Plan.from_network(net.dims, net.tensors, **opts)
    typ = N.typical_magnitude(net.dims, net.tensors)
    mu = plan.sliced()
    val, per = tnq_lib.contract_sliced(plan, per_slice=True)
    ref, ref_per = N.contract_network(net.dims, net.tensors, sliced=mu, per_slice=True)
    assert rel_err(val, ref, typ) < tol, (net.name, val, ref)
    if per_slice:
        slice_typ = typ / np.sqrt(len(ref_per))
        for s in range(len(per)):
            assert rel_err(per[s], ref_per[s], slice_typ) < tol, (net.name, s, per[s], ref_per[s])
    return plan


@pytest.mark.parametrize("L", [3, 5])
def test_lattice_unsliced(cuda, tnq_lib, L):
    """4x4 lattices (bond dimension 3 and 5, padded to 4 and 8 values)."""
    check(tnq_lib, I.random_lattice_network(4, 4, L, seed=L))


@pytest.mark.parametrize("L,p", [(3, 4), (5, 3), (4, 5)])
def test_lattice_sliced_per_slice(cuda, tnq_lib, L, p):
    """5x5 lattices sliced on p binary digits: every slice against the oracle's
    restriction of the same digits (Eq. 4) and the sum (Eq. 5)."""
    net = I.random_lattice_network(5, 5, L, seed=10 + L)
    plan = check(tnq_lib, net, min_p=p, max_p=p)
    assert plan.info()["p"] == p


def test_mixed_dimensions_and_torus(cuda, tnq_lib):
    check(tnq_lib, I.random_lattice_network(4, 5, (2, 3, 5), seed=3), min_p=2, max_p=2)
    check(tnq_lib, I.random_lattice_network(3, 4, 3, seed=4, periodic=True))


@pytest.mark.parametrize("L", [3, 5, 7])
def test_ring_is_the_trace(cuda, tnq_lib, L):
    net = I.random_ring_network(9, L, seed=L)
    plan = tnq_lib.Plan.from_network(net.dims, net.tensors)
    mats = [a for _, a in net.tensors]
    ref = np.trace(np.linalg.multi_dot(mats))
    got = tnq_lib.contract_sliced(plan)
    assert abs(got - ref) <= TOL * max(abs(ref), N.typical_magnitude(net.dims, net.tensors))


@pytest.mark.parametrize("seed", range(6))
def test_degenerate_small_networks(cuda, tnq_lib, seed):
    """Dimension-1 indices (no binary variable), rank-0 scalar tensors, tensors
    whose every variable is sliced, disconnected pieces."""
    net = I.random_small_network(6, 6, 3, dims=(1, 2, 3, 5), seed=200 + seed)
    nvars = sum((d - 1).bit_length() for d in net.dims)
    check(tnq_lib, net, min_p=min(2, nvars), max_p=min(2, nvars))


def test_fused_chains_and_tiles_on_a_larger_lattice(cuda, tnq_lib):
    """A 6x6 lattice at L = 3 whose buckets reach 2^16+ entries: fused chains
    over several tiles and a ragged slice batch."""
    net = I.random_lattice_network(6, 6, 3, seed=21)
    plan = check(tnq_lib, net, min_p=3, max_p=3, fuse_min_rank=10)
    assert plan.info()["n_fused_groups"] > 0
    # a ragged range of slices equals the oracle's partial sum
    mu = plan.sliced()
    got = tnq_lib.contract_sliced(plan, None, 1, 6)
    ref = N.contract_network(net.dims, net.tensors, sliced=mu, slices=(1, 6))
    assert rel_err(got, ref, N.typical_magnitude(net.dims, net.tensors)) < TOL


@pytest.mark.parametrize("precision", [1, 2])
def test_split_precision_network(cuda, tnq_lib, precision):
    net = I.random_lattice_network(5, 5, 4, seed=31)
    plan = tnq_lib.Plan.from_network(net.dims, net.tensors, precision=precision, gemm_min_k_log2=3)
    assert plan.info()["n_gemm_buckets"] > 0
    typ = N.typical_magnitude(net.dims, net.tensors)
    ref = N.contract_network(net.dims, net.tensors)
    assert rel_err(tnq_lib.contract_sliced(plan), ref, typ) < SPLIT_TOL

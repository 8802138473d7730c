"""FP64 oracle for general tensor networks with indices of any dimension L.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg import it; the library's contraction path never does. It shares
no code with the CUDA path (inputs arrive as plain numpy arrays from the
seeded generator).

What it computes (Section II.A: a network's value is the sum, over every
assignment of values to its indices, of the product of the tensor entries the
assignment selects; Eq. 2 eliminates the indices one at a time):

  contract_network(dims, tensors, order=None, sliced=(), slices=None, per_slice=False)

  dims     : dims[i] = L_i >= 1, the number of values of index i
  tensors  : list of (indices, array); `indices` is a tuple of distinct index
             ids and `array` a complex array of shape (dims[i] for i in indices)
             (numpy C order: the first index varies slowest); a tensor with no
             index is a scalar
  order    : elimination order, a permutation of every index id (None: the
             oracle's own greedy min-degree order)
  sliced   : (index, bit) pairs mu_0..mu_{p-1}. Slice s restricts index i to
             the values x whose bit `bit` equals bit j of s, for every
             mu_j = (i, bit) -- Eq. 4 applied to one binary digit of an
             L-valued index (a value x of index i is the digits of x; fixing a
             digit keeps the values that carry it). The 2^p restrictions
             partition the assignments, so the slices sum to the value (Eq. 5).
  slices   : (begin, end) of the slice range, default all 2^p
  Returns the FP64 sum over the slices (increasing s), plus each slice's value
  if per_slice.

Bucket elimination as in Eq. 2: every tensor goes to the bucket of its
earliest index in `order`; in that order, the bucket's tensors are multiplied
as dense arrays over the union of their indices (each broadcast to that
union) and the bucket's index is summed out; the result joins the bucket of
its earliest remaining index, or multiplies the running scalar when it has
none.
"""
from __future__ import annotations

import numpy as np


def _check(dims, tensors):
    n = len(dims)
    for d in dims:
        if int(d) < 1:
            raise ValueError("every index needs at least one value")
    seen = set()
    for idx, arr in tensors:
        if len(set(idx)) != len(idx):
            raise ValueError("a tensor lists an index twice")
        for i in idx:
            if not 0 <= i < n:
                raise ValueError("index id out of range")
            seen.add(i)
        if tuple(np.shape(arr)) != tuple(int(dims[i]) for i in idx):
            raise ValueError("tensor shape does not match its index dimensions")
    if len(seen) != n:
        raise ValueError("every index must appear in some tensor")


def min_degree_order(dims, tensors):
    """Greedy min-degree elimination order of the index interaction graph
    (indices adjacent when they share a tensor); ties to the lowest id."""
    n = len(dims)
    adj = [set() for _ in range(n)]
    for idx, _ in tensors:
        for a in idx:
            for b in idx:
                if a != b:
                    adj[a].add(b)
    left = set(range(n))
    order = []
    while left:
        u = min(left, key=lambda v: (len(adj[v] & left), v))
        nb = adj[u] & left
        for a in nb:
            adj[a] |= nb - {a}
        left.remove(u)
        order.append(u)
    return order


def _restrict(dims, tensors, sliced, s):
    """Slice s of Eq. 4: every tensor holding a sliced index keeps, along that
    index, only the values whose digit `bit` equals bit j of s."""
    out = []
    for idx, arr in tensors:
        a = np.array(arr, dtype=np.complex128)
        for j, (i, bit) in enumerate(sliced):
            if i not in idx:
                continue
            want = (s >> j) & 1
            x = np.arange(int(dims[i]))
            keep = (((x >> bit) & 1) == want).astype(np.float64)
            axis = idx.index(i)
            shape = [1] * a.ndim
            shape[axis] = int(dims[i])
            a = a * keep.reshape(shape)
        out.append((tuple(idx), a))
    return out


def _broadcast(idx, arr, union):
    """The tensor as an array over `union` (size-1 axes where it has no index)."""
    perm = sorted(range(len(idx)), key=lambda k: union.index(idx[k]))
    a = np.transpose(arr, perm) if len(idx) > 1 else arr
    shape = [1] * len(union)
    for k in perm:
        shape[union.index(idx[k])] = arr.shape[k]
    return a.reshape(shape)


def _eliminate(dims, tensors, order):
    """Eq. 2 in the given order: the network's value in FP64."""
    pos = {u: k for k, u in enumerate(order)}
    buckets = {u: [] for u in order}
    scalar = complex(1.0)
    for idx, arr in tensors:
        if len(idx) == 0:
            scalar *= complex(np.asarray(arr).reshape(()))
        else:
            buckets[min(idx, key=pos.__getitem__)].append((tuple(idx), arr))
    for u in order:
        if not buckets[u]:
            continue
        union = sorted({i for idx, _ in buckets[u] for i in idx}, key=pos.__getitem__)
        prod = np.ones([1] * len(union), dtype=np.complex128)
        for idx, arr in buckets[u]:
            prod = prod * _broadcast(idx, arr, union)
        res = prod.sum(axis=union.index(u))
        rest = tuple(i for i in union if i != u)
        if rest:
            buckets[min(rest, key=pos.__getitem__)].append((rest, res))
        else:
            scalar *= complex(res)
    return scalar


def contract_network(dims, tensors, order=None, sliced=(), slices=None, per_slice=False):
    dims = [int(d) for d in dims]
    tensors = [(tuple(int(i) for i in idx), np.asarray(arr, dtype=np.complex128)) for idx, arr in tensors]
    _check(dims, tensors)
    if order is None:
        order = min_degree_order(dims, tensors)
    order = [int(u) for u in order]
    if sorted(order) != list(range(len(dims))):
        raise ValueError("order must list every index once")
    sliced = [(int(i), int(b)) for i, b in sliced]
    for i, b in sliced:
        if not 0 <= i < len(dims) or b < 0 or (1 << b) >= dims[i]:  # digits of values 0..L-1
            raise ValueError("sliced digit outside the index's values")
    p = len(sliced)
    s0, s1 = slices if slices is not None else (0, 1 << p)
    total = complex(0.0)
    per = []
    for s in range(s0, s1):
        v = _eliminate(dims, _restrict(dims, tensors, sliced, s), order)
        per.append(v)
        total += v
    if per_slice:
        return total, np.array(per, dtype=np.complex128)
    return total


def typical_magnitude(dims, tensors):
    """sqrt(E|Z|^2) of a network whose entries are independent with zero mean
    and the given arrays' mean squared magnitudes: E|Z|^2 = sum over the
    assignments of the product of the entries' second moments = prod_i L_i *
    prod_t mean|T_t|^2 (the cross terms vanish). The error floor of a value
    that cancels to far below this scale, like the Porter-Thomas floor of an
    amplitude."""
    m = 1.0
    for d in dims:
        m *= float(d)
    for _, arr in tensors:
        a = np.asarray(arr)
        if a.size:
            m *= float(np.mean(np.abs(a) ** 2))
    return m ** 0.5

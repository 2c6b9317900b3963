"""Bucket (variable) elimination, FP64 (oracle; test only).

App. A of the paper, written from its description: a tensor is a complex
function of Boolean indexes kept sorted by elimination position; ``*``
broadcasts like NumPy; ``reduce_sum`` sums the first axis.  Each initial
factor goes to the bucket of its first index; buckets are processed in order
(product of the bucket, then sum of its variable, Eq. par_sum); a result of
rank > 0 goes to the bucket of its first index, a scalar multiplies into the
result.  Variables left open (outputs without a delta, Eq. psi_x) are never
eliminated: the tensors that reach them are multiplied together at the end,
giving a set of amplitudes at once.

The order is the oracle's own: the vertical order of Sec. IV.A over all
variables (inputs and outputs included -- their deltas make those steps
trivial).  Slicing (fixing a variable and summing the results) is plain
distributivity and is offered for large cases.
Parity: pinned (App. D tau tables and 1/2, 1-D chain of Eqs. 1delim1-2,
state vector, exact Z[omega]; tests/test_oracle_ve.py).
"""
from functools import reduce

import numpy as np

from . import order as O
from . import ugm


class Tensor:
    def __init__(self, indexes, data):
        self.indexes = tuple(indexes)
        self.data = np.asarray(data, dtype=np.complex128)
        assert self.data.ndim == len(self.indexes)

    def rank(self):
        return len(self.indexes)


def _sorted_tensor(f, pos):
    perm = sorted(range(len(f.scope)), key=lambda a: pos[f.scope[a]])
    return Tensor([f.scope[a] for a in perm], np.transpose(f.table, perm))


def multiply(a: Tensor, b: Tensor, pos) -> Tensor:
    """Broadcast product: a missing index acts as a size-1 axis."""
    union = sorted(set(a.indexes) | set(b.indexes), key=lambda v: pos[v])

    def expand(t):
        shape = [2 if v in t.indexes else 1 for v in union]
        return t.data.reshape(shape)

    return Tensor(union, expand(a) * expand(b))


def reduce_sum(t: Tensor) -> Tensor:
    """Sum over the first axis."""
    return Tensor(t.indexes[1:], t.data.sum(axis=0))


def eliminate(factors, order, open_vars=()):
    """Run bucket elimination.  Returns a Tensor over ``open_vars`` (sorted by
    their position after ``order``), a rank-0 Tensor when nothing is open."""
    open_vars = list(open_vars)
    pos = {v: i for i, v in enumerate(list(order) + open_vars)}
    buckets = {v: [] for v in order}
    result = None
    remaining = []

    def place(t):
        nonlocal result
        if t.rank() == 0:
            result = t if result is None else Tensor((), result.data * t.data)
        elif t.indexes[0] in buckets:
            buckets[t.indexes[0]].append(t)
        else:
            remaining.append(t)

    for f in factors:
        place(_sorted_tensor(f, pos))
    for v in order:
        bucket = buckets[v]
        if not bucket:
            continue
        prod = reduce(lambda a, b: multiply(a, b, pos), bucket)
        place(reduce_sum(prod))
    for t in remaining:
        result = t if result is None else multiply(result, t, pos)
    if result is None:
        result = Tensor((), np.complex128(1.0))
    if open_vars:
        # broadcast over open variables that no factor touches
        full = Tensor(open_vars, np.ones([2] * len(open_vars)))
        result = multiply(full, result, pos)
    return result


def vertical_order(model, circuit, open_outputs=False):
    rows, cols = (circuit.rows, circuit.cols) if circuit.rows else (1, model.n)
    allv = list(range(model.n_vars))
    if open_outputs:
        allv = [v for v in allv if v not in set(model.outputs)]
    return O.vertical(model, allv, rows, cols)


def amplitude(circuit, x, model=None, order=None, slice_vars=()) -> complex:
    """<x|C|0^n> by bucket elimination, optionally sliced over ``slice_vars``."""
    m = model or ugm.build(circuit)
    order = order or vertical_order(m, circuit)
    fs = ugm.factors_for(m, x)
    if not slice_vars:
        return complex(eliminate(fs, order).data)
    total = 0.0 + 0.0j
    for s in range(1 << len(slice_vars)):
        extra = [ugm.delta(v, (s >> i) & 1) for i, v in enumerate(slice_vars)]
        total += complex(eliminate(fs + extra, order).data)
    return total


def amplitudes(circuit, xs, order=None) -> np.ndarray:
    m = ugm.build(circuit)
    order = order or vertical_order(m, circuit)
    return np.array([amplitude(circuit, x, m, order) for x in xs])


def open_amplitudes(circuit) -> np.ndarray:
    """All 2^n amplitudes at once: output deltas omitted (Eq. psi_x).
    Entry x has bit j = qubit j."""
    m = ugm.build(circuit)
    order = vertical_order(m, circuit, open_outputs=True)
    # open variables ordered qubit n-1 first so that the flattened C-order
    # index has qubit j at bit j
    open_vars = [m.outputs[j] for j in reversed(range(m.n))]
    t = eliminate(ugm.factors_for(m, open_outputs=True), order, open_vars)
    return t.data.reshape(-1)

"""Pins for oracle/ve.c (FP64 bucket elimination in plain C, App. A) and the
greedy slicer of oracle/order.py."""
import numpy as np
import pytest

import qgm_inputs as qi
from oracle import order as O
from oracle import statevector as sv
from oracle import ugm, ve, vec


def test_app_d_half(app_d):
    # App. D: <00|C|00> = 1/2 for H H, CZ, H H; the other outputs by the
    # state vector (1/2, 1/2, 1/2, -1/2)
    for x, ref in [(0, 0.5), (1, 0.5), (2, 0.5), (3, -0.5)]:
        assert abs(vec.amplitude(app_d, x) - ref) < 1e-15


@pytest.mark.parametrize("rows,cols,depth", [(3, 3, 8), (3, 4, 12), (4, 4, 10), (2, 5, 15)])
def test_state_vector_small_grids(rows, cols, depth):
    c = qi.grid_circuit(rows, cols, depth, 0)
    bits = qi.bitstrings(c.n, 16, 0)
    ref = sv.amplitudes(c, bits)
    a = np.array([vec.amplitude(c, x) for x in bits])
    assert np.max(np.abs(a - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_normalisation_all_outputs():
    # sum_x |<x|C|0>|^2 = 1 over all 2^n outputs (unitarity)
    c = qi.grid_circuit(3, 3, 10, 1)
    m = ugm.build(c)
    pr = vec.Prepared(m)
    order, _ = O.min_fill(O.graph(m))
    p = sum(abs(vec.amplitude(c, x, order=order, model=m, prepared=pr)) ** 2 for x in range(2 ** c.n))
    assert abs(p - 1.0) < 1e-12


def test_parametrised_and_vertical_order():
    c = qi.grid_circuit(3, 3, 9, 2, param=True)
    m = ugm.build(c)
    bits = qi.bitstrings(c.n, 8, 2)
    order = ve.vertical_order(m, c)
    order = [v for v in order if v not in set(m.inputs) | set(m.outputs)]
    a = np.array([vec.amplitude(c, x, order=order) for x in bits])
    assert np.max(np.abs(a - ve.amplitudes(c, bits))) < 1e-14


@pytest.mark.parametrize("n_slices", [1, 3, 6])
def test_sliced_equals_unsliced(n_slices):
    # slicing is distributivity: the sum of the conditioned eliminations
    c = qi.grid_circuit(4, 4, 14, 0)
    m = ugm.build(c)
    adj = O.graph(m)
    order, w = O.min_fill(adj)
    sl = O.slice_greedy(adj, order, n_slices=n_slices)
    assert len(sl) == n_slices and len(set(sl)) == n_slices
    assert max(len(q) for q in O.cliques(adj, order, sl)) < w
    for x in qi.bitstrings(c.n, 4, 0):
        ref = sv.amplitudes(c, [x])[0]
        assert abs(vec.amplitude(c, x, order=order, slice_vars=sl) - ref) < 1e-14


def test_slice_greedy_by_hand():
    # a path a-b-c-d-e eliminated from the middle out: order c, b, d, a, e
    # makes cliques {c,b,d}, {b,a,d}, {d,a,e}, {a,e}, {e}; the largest size is
    # 3 and d lies in all three of them -> d first; without d the cliques are
    # {c,b}, {b,a}, {a}, {e}: b lies in both cliques of size 2 -> b next
    a, b, cc, d, e = 0, 1, 2, 3, 4
    adj = {a: {b}, b: {a, cc}, cc: {b, d}, d: {cc, e}, e: {d}}
    order = [cc, b, d, a, e]
    cl = O.cliques(adj, order)
    assert [sorted(q) for q in cl] == [[1, 2, 3], [0, 1, 3], [0, 3, 4], [0, 4], [4]]
    assert O.slice_greedy(adj, order, n_slices=1) == [d]
    assert O.slice_greedy(adj, order, n_slices=2) == [d, b]
    assert O.slice_greedy(adj, order, max_clique=2) == [d]

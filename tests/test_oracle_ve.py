"""Pins for oracle/ve.py (bucket elimination, App. A)."""
import math

import numpy as np
import pytest

import qgm_inputs as qi
from oracle import gates as G
from oracle import statevector as sv
from oracle import ugm
from oracle import ve


def test_app_d_intermediate_tables(app_d):
    m = ugm.build(app_d)
    # variables: b_0^0=0, b_1^0=1, b_0^1=2, b_1^1=3, b_0^2=4, b_1^2=5
    assert m.n_vars == 6 and m.outputs == [4, 5]
    fs = ugm.factors_for(m, 0)
    # eliminate the four boundary variables first (App. D), then b_1^1, b_0^1
    order = [0, 1, 4, 5, 3, 2]
    pos = {v: i for i, v in enumerate(order)}
    tens = [ve._sorted_tensor(f, pos) for f in fs]
    # bucket elimination of the boundary variables leaves factors on b_0^1, b_1^1
    rest = []
    buckets = {v: [] for v in order}
    for t in tens:
        buckets[t.indexes[0]].append(t)
    for v in order[:4]:
        prod = buckets[v][0]
        for t in buckets[v][1:]:
            prod = ve.multiply(prod, t, pos)
        r = ve.reduce_sum(prod)
        buckets[r.indexes[0]].append(r)
    tau1 = buckets[3][0]
    for t in buckets[3][1:]:
        tau1 = ve.multiply(tau1, t, pos)
    for t in buckets[2]:
        tau1 = ve.multiply(tau1, t, pos)
    # tau_1(b_0^1, b_1^1) = (1/4, 1/4, 1/4, -1/4)
    assert tau1.indexes == (3, 2)
    assert np.allclose(tau1.data, [[0.25, 0.25], [0.25, -0.25]], atol=1e-15)
    tau2 = ve.reduce_sum(tau1)          # sum over b_1^1
    assert np.allclose(tau2.data, [0.5, 0.0], atol=1e-15)
    assert abs(complex(ve.reduce_sum(tau2).data) - 0.5) < 1e-15
    assert abs(ve.amplitude(app_d, 0) - 0.5) < 1e-15


def test_one_dimensional_chain():
    # Eqs. 1delim1-2: a single worldline is a product of 2x2 factors
    Gt = qi.Gate
    kinds = [qi.GATE_H] + [qi.GATE_X12, qi.GATE_T, qi.GATE_Y12, qi.GATE_H] * 5
    c = qi.circuit_from_gates(1, [Gt(k, t, 0) for t, k in enumerate(kinds)])
    U = np.eye(2, dtype=complex)
    for k in kinds:
        U = G.matrix(k) @ U
    for x in (0, 1):
        assert abs(ve.amplitude(c, x) - U[x, 0]) < 1e-14


@pytest.mark.parametrize("rows,cols,depth,seed", [(3, 3, 10, 0), (2, 4, 14, 1), (3, 4, 9, 2)])
def test_ve_equals_state_vector(rows, cols, depth, seed):
    c = qi.grid_circuit(rows, cols, depth, seed)
    xs = qi.bitstrings(c.n, 8, seed)
    assert np.allclose(ve.amplitudes(c, xs), sv.amplitudes(c, xs), atol=1e-14, rtol=0)


def test_ve_parametrised_equals_state_vector():
    c = qi.grid_circuit(3, 3, 12, 7, param=True)
    xs = qi.bitstrings(c.n, 8, 7)
    assert np.allclose(ve.amplitudes(c, xs), sv.amplitudes(c, xs), atol=1e-14, rtol=0)


def test_open_outputs_give_all_amplitudes():
    c = qi.grid_circuit(3, 3, 8, 0)
    assert np.allclose(ve.open_amplitudes(c), sv.state(c), atol=1e-14, rtol=0)


def test_open_outputs_4x4_normalised():
    a = ve.open_amplitudes(qi.grid_circuit(4, 4, 10, 0))
    assert a.size == 1 << 16
    assert abs(np.vdot(a, a).real - 1) < 1e-12


def test_slicing_is_distributive():
    c = qi.grid_circuit(3, 3, 12, 3)
    m = ugm.build(c)
    x = int(qi.bitstrings(c.n, 1, 3)[0])
    free = [v for v in range(m.n_vars) if v not in m.inputs and v not in m.outputs]
    a = ve.amplitude(c, x, m)
    assert abs(ve.amplitude(c, x, m, slice_vars=free[3:6]) - a) < 1e-14

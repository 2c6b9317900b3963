"""Pins for oracle/grad.py."""
import math

import numpy as np
import pytest

import qgm_inputs as qi
from oracle import grad as OG
from oracle import ve


def test_one_qubit_closed_form():
    # a_0 = cos(t/2), a_1 = -i e^{i phi} sin(t/2): L = log cos^2 + log sin^2
    th, ph = 1.1, 0.7
    c = qi.circuit_from_gates(1, [qi.Gate(qi.GATE_RXY, 0, 0, -1, th, ph)])
    g = OG.grad_exact(c, [0, 1])
    assert abs(g[0] - (-math.tan(th / 2) + 1 / math.tan(th / 2))) < 1e-12
    assert abs(g[1]) < 1e-12


@pytest.mark.parametrize("rows,cols,depth,seed", [(2, 3, 10, 1), (3, 3, 9, 2)])
def test_exact_equals_finite_differences(rows, cols, depth, seed):
    c = qi.grid_circuit(rows, cols, depth, seed, param=True)
    xs = qi.bitstrings(c.n, 6, seed)
    g = OG.grad_exact(c, xs)
    fd = OG.grad_fd(c, xs, h=1e-5)
    ref = np.array([fd[q] for q in range(len(g))])
    assert np.max(np.abs(g - ref)) < 1e-6 * max(1.0, np.max(np.abs(ref)))


def test_ve_derivative_matches_state_vector():
    c = qi.grid_circuit(3, 3, 10, 4, param=True)
    x = int(qi.bitstrings(c.n, 1, 4)[0])
    for p in (0, len(c.param_gates) - 1):
        for w in (0, 1):
            gi = c.param_gates[p]
            from oracle import gates as G
            dM = G.drot(c.gates[gi].theta, c.gates[gi].phi)[w]
            ref = OG._state_with(c, gi, dM)[x]
            assert abs(OG.amplitude_derivative_ve(c, x, p, w) - ref) < 1e-14

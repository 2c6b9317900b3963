"""Pins for oracle/statevector.py and oracle/pathsum.py."""
import cmath
import math

import numpy as np
import pytest

import qgm_inputs as qi
from oracle import pathsum as ps
from oracle import statevector as sv


def test_app_d_amplitude_is_one_half(app_d):
    # App. D: <00|C|00> = 1/2 for C = (H x H) CZ (H x H)
    psi = sv.state(app_d)
    assert abs(psi[0] - 0.5) < 1e-15
    assert abs(ps.feynman(app_d, 0) - 0.5) < 1e-15
    assert ps.zomega(app_d, 0) == (4, [2, 0, 0, 0])  # 2^{-2} * 2


@pytest.mark.parametrize("rows,cols,depth", [(3, 3, 12), (2, 5, 16)])
def test_normalisation(rows, cols, depth):
    psi = sv.state(qi.grid_circuit(rows, cols, depth, seed=1))
    assert abs(np.vdot(psi, psi).real - 1) < 1e-12


@pytest.mark.parametrize("rows,cols,depth,seed", [(2, 2, 8, 0), (2, 3, 8, 1), (3, 3, 6, 2)])
def test_state_vector_equals_path_sums(rows, cols, depth, seed):
    c = qi.grid_circuit(rows, cols, depth, seed)
    psi = sv.state(c)
    for x in qi.bitstrings(c.n, 6, seed):
        a = psi[int(x)]
        assert abs(ps.feynman(c, x) - a) < 1e-13
        L, p = ps.zomega(c, x)
        assert abs(ps.zomega_value(L, p) - a) < 1e-13


@pytest.mark.parametrize("rows,cols,depth,seed", [(2, 3, 9, 0), (3, 3, 7, 4)])
def test_appF_ising_form_up_to_constant_phase(rows, cols, depth, seed):
    # App. F drops x-independent phases; reading X^1/2 = exp(-i pi X / 4)
    # each X^1/2 contributes exactly omega^2 = i, so a_F = i^{n_X} a.
    c = qi.grid_circuit(rows, cols, depth, seed)
    psi = sv.state(c)
    n_x = sum(g.kind == qi.GATE_X12 for g in c.gates)
    for x in range(1 << c.n):
        if abs(psi[x]) < 1e-9:
            continue
        assert abs(ps.ising_appF(c, x) - (1j ** n_x) * psi[x]) < 1e-12


def test_clifford_probabilities_are_dyadic():
    # Without T, path phases are multiples of pi/2: probabilities 0 or 2^-k.
    G = qi.Gate
    rng = np.random.default_rng(5)
    gates = [G(qi.GATE_H, 0, q) for q in range(3)]
    for t in range(1, 12):
        a, b = sorted(rng.choice(3, 2, replace=False))
        gates.append(G(qi.GATE_CZ, t, int(a), int(b)))
        c3 = ({0, 1, 2} - {a, b}).pop()
        gates.append(G(int(rng.choice([qi.GATE_X12, qi.GATE_Y12, qi.GATE_H])), t, int(c3)))
    psi = sv.state(qi.circuit_from_gates(3, gates))
    for p in np.abs(psi) ** 2:
        assert p < 1e-14 or abs(math.log2(p) - round(math.log2(p))) < 1e-9


def test_parametrised_matches_fixed_at_special_angles():
    c = qi.grid_circuit(2, 3, 10, seed=0, param=True)
    f = qi.grid_circuit(2, 3, 10, seed=0)
    th = [math.pi / 2] * len(c.param_gates)
    ph = [0.0 if f.gates[i].kind == qi.GATE_X12 else math.pi / 2 for i in c.param_gates]
    assert np.allclose(sv.state(c.with_angles(th, ph)), sv.state(f), atol=1e-14)

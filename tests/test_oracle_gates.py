"""Pins for oracle/gates.py: definitions of the gate set (paper Sec. II) and
App. D's psi tables, checked against scipy's matrix exponential."""
import math

import numpy as np
import pytest
import scipy.linalg as sl

from oracle import gates as G


def test_unitary():
    for U in (G.H, G.X12, G.Y12, G.T, G.rot(1.1, 0.3)):
        assert np.allclose(U.conj().T @ U, np.eye(2), atol=1e-15)


def test_rotations_are_pi_over_2_about_x_and_y():
    assert np.allclose(G.X12, sl.expm(-1j * math.pi / 4 * G.PX), atol=1e-15)
    assert np.allclose(G.Y12, sl.expm(-1j * math.pi / 4 * G.PY), atol=1e-15)
    # two half rotations are a full pi rotation: exp(-i pi X / 2) = -i X
    assert np.allclose(G.X12 @ G.X12, -1j * G.PX, atol=1e-15)
    assert np.allclose(G.Y12 @ G.Y12, -1j * G.PY, atol=1e-15)


@pytest.mark.parametrize("theta,phi", [(0.3, 0.0), (1.9, 2.5), (2.7, 5.9)])
def test_parametrised_gate_is_exponential(theta, phi):
    gen = math.cos(phi) * G.PX + math.sin(phi) * G.PY
    assert np.allclose(G.rot(theta, phi), sl.expm(-0.5j * theta * gen), atol=1e-14)
    dth, dph = G.drot(theta, phi)
    h = 1e-6
    fd_th = (G.rot(theta + h, phi) - G.rot(theta - h, phi)) / (2 * h)
    fd_ph = (G.rot(theta, phi + h) - G.rot(theta, phi - h)) / (2 * h)
    assert np.allclose(dth, fd_th, atol=1e-9) and np.allclose(dph, fd_ph, atol=1e-9)


def test_special_angles_reduce_to_fixed_gates():
    assert np.allclose(G.rot(math.pi / 2, 0), G.X12, atol=1e-15)
    assert np.allclose(G.rot(math.pi / 2, math.pi / 2), G.Y12, atol=1e-15)


def test_app_d_tables_and_t_gate():
    # App. D: psi_H(1,1) = -1/sqrt2, others +1/sqrt2; psi_CZ(1,1) = -1, others 1
    s = 1 / math.sqrt(2)
    assert np.allclose(G.H, [[s, s], [s, -s]])
    assert np.allclose(G.CZ_DIAG, [[1, 1], [1, -1]])
    # T = diag(1, e^{i pi / 4})
    assert np.allclose(G.T, np.diag([1, np.exp(1j * math.pi / 4)]))

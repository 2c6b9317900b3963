"""Gate matrices, FP64, written from their definitions (oracle; test only).

Paper, Sec. "Numerical results": H is the Hadamard; X^1/2 (Y^1/2) is a pi/2
rotation about the X (Y) axis of the Bloch sphere; T = diag(1, e^{i pi/4});
CZ = diag(1, 1, 1, -1).  The rotation sign is fixed as exp(-i pi X/4), the
reading under which App. F's X^1/2 phase term (Eq. phX) holds.  The
parametrised gate is exp(-i theta (cos phi X + sin phi Y)/2), which is X^1/2
at (pi/2, 0) and Y^1/2 at (pi/2, pi/2).

Matrix convention: ``U[out, in]`` = <out|U|in>, the factor psi_U(b', b) of
Sec. III.B with b' the state after the gate.
Parity: pinned (tests/test_oracle_gates.py: unitarity, scipy expm of the
generator, App. D tables).
"""
import math

import numpy as np

SQ2 = 1.0 / math.sqrt(2.0)
I2 = np.eye(2, dtype=np.complex128)
PX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
PZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def rot(theta: float, phi: float) -> np.ndarray:
    """exp(-i theta n.sigma / 2) with n = (cos phi, sin phi, 0).

    Since (n.sigma)^2 = 1 the exponential is cos(theta/2) I - i sin(theta/2) n.sigma.
    """
    ns = math.cos(phi) * PX + math.sin(phi) * PY
    return math.cos(theta / 2) * I2 - 1j * math.sin(theta / 2) * ns


def drot(theta: float, phi: float):
    """(d/dtheta, d/dphi) of rot(theta, phi)."""
    ns = math.cos(phi) * PX + math.sin(phi) * PY
    dns = -math.sin(phi) * PX + math.cos(phi) * PY
    d_theta = -0.5 * math.sin(theta / 2) * I2 - 0.5j * math.cos(theta / 2) * ns
    d_phi = -1j * math.sin(theta / 2) * dns
    return d_theta, d_phi


H = SQ2 * np.array([[1, 1], [1, -1]], dtype=np.complex128)
X12 = rot(math.pi / 2, 0.0)
Y12 = rot(math.pi / 2, math.pi / 2)
T = np.diag([1.0, np.exp(1j * math.pi / 4)]).astype(np.complex128)
CZ_DIAG = np.array([[1, 1], [1, -1]], dtype=np.complex128)  # psi_CZ(b, b')


def matrix(kind: int, theta: float = 0.0, phi: float = 0.0) -> np.ndarray:
    """2x2 matrix of a one-qubit gate kind (see qgm_inputs for kind ids)."""
    if kind == 0:
        return H
    if kind == 1:
        return X12
    if kind == 2:
        return Y12
    if kind == 3:
        return T
    if kind == 5:
        return rot(theta, phi)
    raise ValueError(f"not a one-qubit gate kind: {kind}")


def is_diagonal(kind: int) -> bool:
    """T and CZ keep the computational basis state (Sec. III.A)."""
    return kind in (3, 4)

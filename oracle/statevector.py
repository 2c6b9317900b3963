"""FP64 state vector (oracle; test only).

a_x = <x|C|0^n>: the gate unitaries applied cycle by cycle to |0^n>, which is
what the path sum of Eq. fpath adds up.  Bit j of the index x is qubit j.
Used for n <= ~25 (2^25 complex128 = 512 MiB).
Parity: pinned (App. D worked example 1/2, normalisation, brute-force path
sum and the exact Z[omega] form on tiny circuits; tests/test_oracle_sv.py).
"""
import numpy as np

from . import gates as G


def apply_1q(psi: np.ndarray, n: int, q: int, U: np.ndarray) -> np.ndarray:
    v = psi.reshape(1 << (n - 1 - q), 2, 1 << q)
    out = np.einsum("ab,ibj->iaj", U, v)
    return out.reshape(-1)


def apply_cz(psi: np.ndarray, n: int, a: int, b: int) -> np.ndarray:
    idx = np.arange(psi.size, dtype=np.int64)
    mask = ((idx >> a) & 1) & ((idx >> b) & 1)
    out = psi.copy()
    out[mask == 1] *= -1.0
    return out


def state(circuit) -> np.ndarray:
    """Final state C|0^n> as a complex128 vector of length 2^n."""
    n = circuit.n
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    for g in circuit.gates:
        if g.kind == 4:
            psi = apply_cz(psi, n, g.q0, g.q1)
        else:
            psi = apply_1q(psi, n, g.q0, G.matrix(g.kind, g.theta, g.phi))
    return psi


def amplitudes(circuit, xs) -> np.ndarray:
    psi = state(circuit)
    return psi[np.asarray(xs, dtype=np.int64)]

"""Expectation values <0|U^dagger O U|0> of Pauli strings (oracle; test only).

Sec. III of the paper: the expectation of an operator O follows the same
method as an amplitude, after cancelling U_a^dagger U_a wherever possible for
a local O.  The oracle computes it from the definition: the FP64 state
vector psi = U|0^n> and <psi|P|psi> with P the tensor product of the Pauli
matrices named by the string (character j acts on qubit j: I, X, Y or Z).
``light_cone`` lists the gates that cannot cancel: scanning from the last
gate back, a gate on a qubit of the current support stays and adds its
qubits to the support; every other gate meets its inverse and drops out.
Parity: pinned (closed forms for H|0>, X^1/2|0>, Y^1/2|0> and a Bell pair;
the purity sum over all Pauli strings of a pure state; <Z_j> from the
probabilities; tests/test_oracle_observable.py).
"""
import numpy as np

from . import gates as G
from . import statevector as sv

PAULI = {"I": np.eye(2, dtype=np.complex128), "X": G.PX, "Y": G.PY, "Z": G.PZ}


def expectation(circuit, pauli: str) -> complex:
    if len(pauli) != circuit.n:
        raise ValueError("one Pauli character per qubit")
    psi = sv.state(circuit)
    phi = psi
    for j, ch in enumerate(pauli):
        if ch != "I":
            phi = sv.apply_1q(phi, circuit.n, j, PAULI[ch])
    return complex(np.vdot(psi, phi))


def light_cone(circuit, pauli: str):
    support = {j for j, ch in enumerate(pauli) if ch != "I"}
    keep = []
    for gi in range(len(circuit.gates) - 1, -1, -1):
        g = circuit.gates[gi]
        qs = {g.q0} if g.q1 < 0 else {g.q0, g.q1}
        if qs & support:
            keep.append(gi)
            support |= qs
    return sorted(keep), sorted(support)

"""Expectation values <0|U^dagger P U|0> of Pauli strings (Sec. III).

The library cancels the gates outside P's backward light cone and writes
the rest as the circuit W = V, P, V^dagger (qgm_circuit_observable); the
expectation is phase * <0|W|0>, one amplitude of W, computed on the GPU by a
plan like any other.
"""
import numpy as np

from ._lib import EXEC_AUTO, Model, Plan


def expectation(circuit, pauli: str, executor=EXEC_AUTO, order_kind=0) -> complex:
    """<0|U^dagger P U|0> for the library circuit `circuit` and Pauli string
    `pauli` (character j acts on qubit j)."""
    w, phase, _ = circuit.observable(pauli)
    if w is None:
        return complex(phase)
    plan = Plan(Model(w), batch=1, executor=executor, order_kind=order_kind).bind()
    a = plan.amplitudes_host(np.zeros(1, dtype=np.uint64))[0]
    return complex(phase * a)

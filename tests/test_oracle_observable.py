"""Pins for oracle/observable.py (expectation values, Sec. III)."""
import itertools
import math

import numpy as np
import pytest

import qgm_inputs as qi
from oracle import observable as OB
from oracle import statevector as sv

G = qi.Gate


def one(kind):
    return qi.circuit_from_gates(1, [G(kind, 0, 0)])


def test_closed_forms_single_qubit():
    # H|0> = |+>: <X> = 1; X^1/2|0> = (|0> - i|1>)/sqrt2: <Y> = -1;
    # Y^1/2|0> = (|0> + |1>)/sqrt2: <X> = 1; |0> itself: <Z> = 1
    assert abs(OB.expectation(one(qi.GATE_H), "X") - 1) < 1e-12
    assert abs(OB.expectation(one(qi.GATE_H), "Z")) < 1e-12
    assert abs(OB.expectation(one(qi.GATE_X12), "Y") + 1) < 1e-12
    assert abs(OB.expectation(one(qi.GATE_Y12), "X") - 1) < 1e-12
    assert abs(OB.expectation(one(qi.GATE_T), "Z") - 1) < 1e-12


def test_bell_pair():
    # H on both, CZ, H on qubit 1: (|00> + |11>)/sqrt2 -> <ZZ> = <XX> = 1, <YY> = -1, <Z I> = 0
    c = qi.circuit_from_gates(2, [G(qi.GATE_H, 0, 0), G(qi.GATE_H, 0, 1), G(qi.GATE_CZ, 1, 0, 1),
                                  G(qi.GATE_H, 2, 1)])
    assert abs(OB.expectation(c, "ZZ") - 1) < 1e-12
    assert abs(OB.expectation(c, "XX") - 1) < 1e-12
    assert abs(OB.expectation(c, "YY") + 1) < 1e-12
    assert abs(OB.expectation(c, "ZI")) < 1e-12


def test_purity_sum_over_all_pauli_strings():
    # a pure state has sum_P <P>^2 = 2^n over the 4^n Pauli strings, each <P> real
    c = qi.grid_circuit(1, 3, 6, 4)
    vals = [OB.expectation(c, "".join(p)) for p in itertools.product("IXYZ", repeat=3)]
    assert max(abs(v.imag) for v in vals) < 1e-12
    assert abs(sum(v.real ** 2 for v in vals) - 8) < 1e-10


def test_z_from_probabilities():
    c = qi.grid_circuit(2, 3, 8, 1)
    p = np.abs(sv.state(c)) ** 2
    x = np.arange(p.size)
    for j in range(c.n):
        pauli = "".join("Z" if i == j else "I" for i in range(c.n))
        assert abs(OB.expectation(c, pauli) - np.sum(p * (1 - 2 * ((x >> j) & 1)))) < 1e-12


def test_light_cone_drops_gates_that_cancel():
    # the expectation on the light-cone circuit alone equals the full one
    c = qi.grid_circuit(3, 3, 5, 2)
    pauli = "IIIIZIIII"
    keep, support = OB.light_cone(c, pauli)
    assert len(keep) < len(c.gates)
    sub = qi.circuit_from_gates(c.n, [c.gates[i] for i in keep])
    assert abs(OB.expectation(sub, pauli) - OB.expectation(c, pauli)) < 1e-12

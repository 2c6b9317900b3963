"""Brute-force path sums (oracle; test only).

* ``feynman``: Eq. psi_x summed term by term -- every assignment of the
  variables that are not fixed by the boundary deltas, product of all factor
  values.  Exponential; for <= ~22 free variables.
* ``zomega``: the same sum done exactly.  Every factor of the fixed gate set is
  2^{-1/2} omega^k (non-diagonal) or omega^k (T, CZ) with omega = e^{i pi/4}
  (App. F: all paths have modulus 2^{-L/2} and a phase in multiples of pi/4),
  so a_x = 2^{-L/2} * sum_k c_k omega^k with integer path counts c_k.
* ``ising_appF``: App. F's Ising form, Eqs. path1, phX, phT, phCZ, with spins
  s = 1 - 2b.  Its constant phases are dropped by the paper, so it equals a_x
  up to a unit factor that does not depend on x.

Parity: pinned (tests/test_oracle_sv.py compares the three with each other and
with the state vector; App. D gives 1/2).
"""
import cmath
import math

import numpy as np

from . import ugm

OMEGA = cmath.exp(1j * math.pi / 4)


def _free_vars(model, open_outputs):
    fixed = set(model.inputs)
    if not open_outputs:
        fixed |= set(model.outputs)
    return [v for v in range(model.n_vars) if v not in fixed]


def _assignments(model, x, free):
    """Array [2^F, n_vars] of variable values for every path."""
    F = len(free)
    idx = np.arange(1 << F, dtype=np.int64)
    vals = np.zeros((1 << F, model.n_vars), dtype=np.int64)
    for i, v in enumerate(free):
        vals[:, v] = (idx >> i) & 1
    for j, v in enumerate(model.outputs):
        if v not in free:
            vals[:, v] = (int(x) >> j) & 1
    return vals


def feynman(circuit, x) -> complex:
    """Sum over all paths of the product of the gate factors (Eq. psi_x)."""
    m = ugm.build(circuit)
    free = _free_vars(m, False)
    if len(free) > 24:
        raise ValueError("too many free variables for brute force")
    vals = _assignments(m, x, free)
    prod = np.ones(vals.shape[0], dtype=np.complex128)
    for f in m.factors:
        prod *= f.table[tuple(vals[:, v] for v in f.scope)]
    return complex(prod.sum())


def _phase_table(kind, scope_len):
    """Phase exponents k (value = [2^{-1/2}] omega^k) of a fixed gate factor,
    read off the gate matrices: H -> 4 b b'; X^1/2 -> 6 [b != b'];
    Y^1/2 -> 4 [b' = 0 and b = 1]; T -> b; CZ -> 4 b b'."""
    if kind == 0:
        return np.array([[0, 0], [0, 4]])
    if kind == 1:
        return np.array([[0, 6], [6, 0]])
    if kind == 2:
        return np.array([[0, 4], [0, 0]])
    if kind == 3:
        return np.array([0, 1])
    if kind == 4:
        return np.array([[0, 0], [0, 4]])
    raise ValueError("parametrised gates have no exact Z[omega] form")


def zomega(circuit, x):
    """Exact a_x as (L, p) with a_x = 2^{-L/2} (p0 + p1 w + p2 w^2 + p3 w^3)."""
    m = ugm.build(circuit)
    free = _free_vars(m, False)
    if len(free) > 24:
        raise ValueError("too many free variables for brute force")
    vals = _assignments(m, x, free)
    phase = np.zeros(vals.shape[0], dtype=np.int64)
    for f in m.factors:
        g = circuit.gates[f.gate]
        tab = _phase_table(g.kind, len(f.scope))
        phase += tab[tuple(vals[:, v] for v in f.scope)]
    counts = np.bincount(phase % 8, minlength=8).astype(np.int64)
    p = [int(counts[k] - counts[k + 4]) for k in range(4)]   # omega^4 = -1
    return m.n_nondiag, p


def zomega_value(L, p) -> complex:
    z = sum(p[k] * OMEGA ** k for k in range(4))
    return z * 2.0 ** (-L / 2)


def ising_appF(circuit, x) -> complex:
    """App. F: 2^{-L/2} sum_s exp(i pi H_s(x)/4), spins s = 1 - 2b.

    Readings: the X/Y sums of Eq. phX run over the X^1/2 and Y^1/2 gates only
    (the H of cycle 0 acts on b = 0 and adds no phase), gate k acting between
    s^{k-1} and s^k; d(j, t) counts the non-diagonal gates on qubit j in
    cycles 0..t, so a T or CZ in cycle t acts on s_j^{d(j,t)}.
    """
    m = ugm.build(circuit)
    free = _free_vars(m, False)
    vals = _assignments(m, x, free)
    s = 1 - 2 * vals                       # spins
    phase_over_pi = np.zeros(vals.shape[0], dtype=np.float64)   # (pi/4) H_s / pi
    cur = list(range(m.n))
    nxt = m.n
    for g in circuit.gates:
        if g.kind in (0, 1, 2):
            new = nxt
            nxt += 1
            if g.kind == 1:      # alpha = 1: (i pi / 2) (1 + s^{k-1} s^k) / 2
                phase_over_pi += 0.5 * (1 + s[:, cur[g.q0]] * s[:, new]) / 2
            elif g.kind == 2:    # alpha = 0: i pi (1 - s^{k-1})/2 (1 + s^k)/2
                phase_over_pi += (1 - s[:, cur[g.q0]]) / 2 * (1 + s[:, new]) / 2
            cur[g.q0] = new
        elif g.kind == 3:        # (i pi / 4) (1 - s)/2
            phase_over_pi += 0.25 * (1 - s[:, cur[g.q0]]) / 2
        elif g.kind == 4:        # i pi (1 - s_i)/2 (1 - s_j)/2
            phase_over_pi += (1 - s[:, cur[g.q0]]) / 2 * (1 - s[:, cur[g.q1]]) / 2
        else:
            raise ValueError("App. F covers the fixed gate set only")
    terms = np.exp(1j * math.pi * phase_over_pi)
    return complex(terms.sum()) * 2.0 ** (-m.n_nondiag / 2)

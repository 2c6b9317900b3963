"""The complex undirected graphical model of a circuit (oracle; test only).

Sec. III.A-B of the paper, Eq. psi_x: one Boolean variable b_j^k per qubit j
and per non-diagonal gate k on it (k = 0 is the input value, k = d_j the
output value, Eq. bc), so a qubit has d_j + 1 variables.  Factors:

* non-diagonal one-qubit gate U on qubit j: psi_U(b_j^k, b_j^{k-1}) = <b'|U|b>;
* diagonal one-qubit gate (T): psi_T(b_j^k) on the current variable;
* CZ: psi_CZ(b_i, b_j) on the two current variables (diagonal, no new vertex);
* boundary deltas delta(b_j^0, 0) and, unless the output is left open,
  delta(b_j^{d_j}, x_j).

Variable ids follow creation order: the n input variables b_j^0 first (id j),
then one id per non-diagonal gate in gate-list order.  The same numbering is
the library's convention, so elimination orders can be compared id by id.
Parity: pinned through the worked example of App. D and the path sums.
"""
from dataclasses import dataclass
from typing import List, Tuple

import numpy as np

from . import gates as G


@dataclass
class Factor:
    scope: Tuple[int, ...]     # variable ids, axis order of ``table``
    table: np.ndarray          # complex128, one axis of size 2 per scope var
    gate: int = -1             # index of the gate in the circuit (-1: delta)


@dataclass
class Model:
    n: int
    n_vars: int
    var_qubit: List[int]
    var_k: List[int]
    inputs: List[int]          # b_j^0
    outputs: List[int]         # b_j^{d_j}
    factors: List[Factor]      # gate factors only (no deltas)
    n_nondiag: int             # L of App. F

    def qubit_vars(self, j):
        return [v for v in range(self.n_vars) if self.var_qubit[v] == j]


def build(circuit) -> Model:
    n = circuit.n
    cur = list(range(n))
    var_qubit = list(range(n))
    var_k = [0] * n
    nv = n
    factors: List[Factor] = []
    L = 0
    for gi, g in enumerate(circuit.gates):
        if g.kind == 4:
            factors.append(Factor((cur[g.q0], cur[g.q1]), G.CZ_DIAG.copy(), gi))
        elif G.is_diagonal(g.kind):
            U = G.matrix(g.kind, g.theta, g.phi)
            factors.append(Factor((cur[g.q0],), np.diag(U).copy(), gi))
        else:
            U = G.matrix(g.kind, g.theta, g.phi)
            v = nv
            nv += 1
            var_qubit.append(g.q0)
            var_k.append(var_k[cur[g.q0]] + 1)
            # psi_U(b', b) with b' the new variable: axis 0 = new, axis 1 = old
            factors.append(Factor((v, cur[g.q0]), U.copy(), gi))
            cur[g.q0] = v
            L += 1
    return Model(n, nv, var_qubit, var_k, list(range(n)), list(cur), factors, L)


def delta(v: int, value: int) -> Factor:
    t = np.zeros(2, dtype=np.complex128)
    t[value] = 1.0
    return Factor((v,), t)


def factors_for(model: Model, x=None, open_outputs=False) -> List[Factor]:
    """Gate factors plus the boundary deltas of Eq. psi_x for output x."""
    fs = list(model.factors)
    fs += [delta(v, 0) for v in model.inputs]
    if not open_outputs:
        for j, v in enumerate(model.outputs):
            fs.append(delta(v, (int(x) >> j) & 1))
    return fs

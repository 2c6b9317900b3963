"""Gradients of the log-probability loss, FP64 (oracle; test only).

L = sum_x log |a_x|^2 over a set of output bitstrings (the cross-entropy
estimator of App. B, Eq. cee, up to sign and 1/m), as a function of the angles
(theta_g, phi_g) of the parametrised one-qubit gates.  For real L of the
amplitudes, dL/dp = 2 Re sum_x conj(dL/d conj a_x) da_x/dp with
dL/d conj a_x = a_x / |a_x|^2.

* ``grad_exact``: da_x/dp by derivative insertion -- the state vector run
  again with gate g replaced by its derivative matrix (the circuit is linear
  in each gate).
* ``grad_fd``: central finite differences of L (step h).
* ``amplitude_derivative_ve``: da_x/dp with the derivative matrix inserted,
  by the oracle's bucket elimination (for circuits too wide for a state
  vector).
Parity: pinned (1-qubit closed form; exact vs finite differences;
tests/test_oracle_grad.py).
"""
import numpy as np

from . import gates as G
from . import statevector as sv
from . import ve


def loss(circuit, xs) -> float:
    a = sv.amplitudes(circuit, xs)
    return float(np.sum(np.log(np.abs(a) ** 2)))


def params(circuit):
    th = np.array([circuit.gates[i].theta for i in circuit.param_gates])
    ph = np.array([circuit.gates[i].phi for i in circuit.param_gates])
    return th, ph


def _state_with(circuit, gi, M):
    """Final state with gate ``gi`` replaced by the 2x2 matrix M."""
    n = circuit.n
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    for i, g in enumerate(circuit.gates):
        if g.kind == 4:
            psi = sv.apply_cz(psi, n, g.q0, g.q1)
        else:
            U = M if i == gi else G.matrix(g.kind, g.theta, g.phi)
            psi = sv.apply_1q(psi, n, g.q0, U)
    return psi


def grad_exact(circuit, xs, weights=None):
    """dL/d(theta_p, phi_p) interleaved [th0, ph0, th1, ph1, ...]."""
    xs = np.asarray(xs, dtype=np.int64)
    a = sv.amplitudes(circuit, xs)
    gbar = a / np.abs(a) ** 2 if weights is None else np.asarray(weights)
    out = np.zeros(2 * len(circuit.param_gates))
    for p, gi in enumerate(circuit.param_gates):
        g = circuit.gates[gi]
        for w, dM in enumerate(G.drot(g.theta, g.phi)):
            da = _state_with(circuit, gi, dM)[xs]
            out[2 * p + w] = 2 * np.real(np.sum(np.conj(gbar) * da))
    return out


def grad_fd(circuit, xs, h=1e-4, which=None):
    """Central differences of L; ``which`` restricts to some parameter indices."""
    th, ph = params(circuit)
    idx = range(2 * len(th)) if which is None else which
    out = {}
    for q in idx:
        p, w = divmod(q, 2)
        vals = []
        for s in (+1, -1):
            t2, p2 = th.copy(), ph.copy()
            (t2 if w == 0 else p2)[p] += s * h
            vals.append(loss(circuit.with_angles(t2, p2), xs))
        out[q] = (vals[0] - vals[1]) / (2 * h)
    return out


def amplitude_derivative_ve(circuit, x, p, which):
    """da_x/dtheta_p (which = 0) or /dphi_p (which = 1) by bucket elimination
    with the derivative matrix inserted for parametrised gate p."""
    from . import ugm
    gi = circuit.param_gates[p]
    g = circuit.gates[gi]
    dM = G.drot(g.theta, g.phi)[which]
    m = ugm.build(circuit)
    fs = []
    for f in ugm.factors_for(m, x):
        if f.gate == gi:
            f = ugm.Factor(f.scope, dM.copy(), gi)
        fs.append(f)
    order = ve.vertical_order(m, circuit)
    return complex(ve.eliminate(fs, order).data)

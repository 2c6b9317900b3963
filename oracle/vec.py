"""FP64 bucket elimination in plain C (oracle; test only): ctypes wrapper of
``oracle/ve.c`` (App. A of the paper; see that file's header).

``amplitude(c, x, order, slice_vars)`` computes <x|C|0^n> by eliminating the
free variables of the graphical model (Sec. III) in ``order``; the inputs are
fixed to 0 and the outputs to the bits of x (the deltas of Eq. psi_x), and
the sum over each assignment of ``slice_vars`` is taken here, one elimination
per assignment (distributivity).  The model and its factor tables come from
``oracle.ugm``; the order and the slice variables from ``oracle.order``.
It exists for the circuits the numpy elimination cannot hold (5x9 depth 40):
each bucket's product-sum is a loop over its output entries, so only tensors
of the order's cliques are ever stored.
``amplitude_derivative(c, x, p, which)``: d<x|C|0>/d(theta_p or phi_p) by
derivative insertion (the circuit is linear in each gate: the amplitude with
gate p's table replaced by the derivative of its matrix).
Parity: pinned (App. D 1/2; the state vector on small grids; the numpy
elimination; derivative insertion against the state-vector oracle's;
tests/test_oracle_vec.py).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from . import gates as G
from . import order as O
from . import ugm

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ve.c")
LIB = os.path.join(HERE, "libve.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ve.c into oracle/libve.so (gcc, OpenMP)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) > os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fcx-limited-range", "-shared", "-fPIC", "-o", tmp, SRC]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("gcc failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.c_void_p
        L.ve_amplitude.argtypes = [C.c_int, C.c_int, P, P, P, P, P, P, P, C.c_int, C.c_int, P]
        L.ve_amplitude.restype = C.c_int
        _lib = L
    return _lib


class Prepared:
    """The model's factor tables in the flat arrays ve.c reads."""

    def __init__(self, model):
        self.model = model
        fs = model.factors
        self.rank = np.array([len(f.scope) for f in fs], dtype=np.int32)
        self.off = np.zeros(len(fs), dtype=np.int64)
        self.toff = np.zeros(len(fs), dtype=np.int64)
        o = t = 0
        for i, f in enumerate(fs):
            self.off[i] = o
            self.toff[i] = t
            o += len(f.scope)
            t += 1 << len(f.scope)
        self.vars = np.array([v for f in fs for v in f.scope] or [0], dtype=np.int32)
        tab = np.concatenate([np.asarray(f.table, dtype=np.complex128).reshape(-1) for f in fs])
        self.tables = np.ascontiguousarray(np.stack([tab.real, tab.imag], axis=1).reshape(-1))


def free_graph(model):
    """Interaction graph of the free variables (inputs and outputs fixed)."""
    return O.graph(model)


def amplitude(circuit, x, order=None, slice_vars=(), model=None, prepared=None, threads=0) -> complex:
    """<x|C|0^n> by App. A bucket elimination in FP64, sliced over
    ``slice_vars`` (default order: the oracle's min-fill)."""
    m = model or ugm.build(circuit)
    pr = prepared or Prepared(m)
    if order is None:
        order, _ = O.min_fill(free_graph(m))
    slice_vars = list(slice_vars)
    fixed = np.full(m.n_vars, -1, dtype=np.int32)
    for v in m.inputs:
        fixed[v] = 0
    for j, v in enumerate(m.outputs):
        if v in m.inputs and (int(x) >> j) & 1:
            return 0j  # a qubit without gates keeps its input 0
        fixed[v] = (int(x) >> j) & 1
    elim = np.array([v for v in order if v not in set(slice_vars)], dtype=np.int32)
    total = 0j
    out = np.zeros(2)
    for s in range(1 << len(slice_vars)):
        for i, v in enumerate(slice_vars):
            fixed[v] = (s >> i) & 1
        rc = lib().ve_amplitude(m.n_vars, len(m.factors), pr.rank.ctypes.data, pr.off.ctypes.data,
                                pr.vars.ctypes.data, pr.toff.ctypes.data, pr.tables.ctypes.data,
                                fixed.ctypes.data, elim.ctypes.data, len(elim), threads, out.ctypes.data)
        if rc != 0:
            raise RuntimeError("ve_amplitude: a free variable is missing from the order")
        total += complex(out[0], out[1])
    return total


def amplitude_derivative(circuit, x, p, which, order=None, model=None, prepared=None, threads=0) -> complex:
    """d<x|C|0>/d theta_p (which = 0) or d phi_p (which = 1) for the p-th
    parametrised gate (circuit.param_gates order): the elimination with that
    gate's factor table replaced by its derivative matrix."""
    m = model or ugm.build(circuit)
    pr = prepared or Prepared(m)
    gi = circuit.param_gates[p]
    fi = next(i for i, f in enumerate(m.factors) if f.gate == gi)
    g = circuit.gates[gi]
    dM = np.asarray(G.drot(g.theta, g.phi)[which], dtype=np.complex128).reshape(-1)
    saved = pr.tables.copy()
    t0 = 2 * int(pr.toff[fi])
    pr.tables[t0:t0 + 8] = np.stack([dM.real, dM.imag], axis=1).reshape(-1)
    try:
        return amplitude(circuit, x, order=order, model=m, prepared=pr, threads=threads)
    finally:
        pr.tables[:] = saved


def amplitudes_parallel(circuit, xs, order=None, model=None, prepared=None, workers=0):
    """<x|C|0^n> for every x of ``xs``, one elimination per bitstring on a
    pool of ``workers`` host threads (default: every core), each elimination
    single-threaded (the C call releases the GIL)."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    m = model or ugm.build(circuit)
    pr = prepared or Prepared(m)
    if order is None:
        order, _ = O.min_fill(free_graph(m))
    workers = workers or os.cpu_count() or 1
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return np.array(list(ex.map(lambda x: amplitude(circuit, int(x), order=order, model=m, prepared=pr,
                                                        threads=1), xs)))

"""Seeded synthetic inputs shared by the CUDA path's tests and by the oracle.

This module only *generates inputs*: gate lists of random grid circuits and
output bitstrings.  It holds none of the amplitude arithmetic of the method
(no gate matrices, no factors, no contraction), so that the oracle and the
product path stay independent while reading the very same circuits.

Circuit family (Sec. "Numerical results" of the paper, gate set {H, X^1/2,
Y^1/2, T} plus CZ; the layout rules themselves are only cited there, so the
rules below are this library's written reading of them):

* cycle 0: H on every qubit (the paper's footnote: depth 1 is the H layer);
* cycle t >= 1: CZ on the pairs of pattern ``P[(t-1) mod 8]`` from the fixed
  rotation [HZ0, HZ2, VT0, VT2, HZ1, HZ3, VT1, VT3]; a qubit that was in a CZ
  in cycle t-1 and is in none in cycle t gets one single-qubit gate in cycle
  t: T the first time, afterwards X^1/2 or Y^1/2 drawn uniformly;
* qubit q = r*cols + c; HZ_o pairs (r,c)-(r,c+1) when c = o + 2(r mod 2)
  (mod 4); VT_o pairs (r,c)-(r+1,c) when r = o + 2(c mod 2) (mod 4).  No qubit
  is in two CZs of one cycle (the paper's restriction on neighbouring CZs).
* depth d counts every cycle including the H cycle (Eq. fpath runs over
  t = 0..d-1); there is no final H layer.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written here from its
published definition.  Stream 1 (seed s) gives one draw per X/Y slot in
(cycle, qubit) order, top bit 0 -> X^1/2, 1 -> Y^1/2; in parametrised mode
each such slot instead takes two draws u1, u2 = (r >> 11) * 2^-53 and becomes
RXY(theta = pi*u1, phi = 2*pi*u2).  Stream 2 (seed s + 1) gives the
bitstrings, one draw each, x = r >> (64 - n) (bit j of x is qubit j).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

GATE_H = 0
GATE_X12 = 1
GATE_Y12 = 2
GATE_T = 3
GATE_CZ = 4
GATE_RXY = 5
GATE_NAMES = {GATE_H: "H", GATE_X12: "X^1/2", GATE_Y12: "Y^1/2", GATE_T: "T",
              GATE_CZ: "CZ", GATE_RXY: "RXY"}

_M64 = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64:
    """SplitMix64 generator: state advances by the golden-ratio increment,
    the output is the state passed through two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next(self) -> int:
        self.state = (self.state + _GOLDEN) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits of one draw."""
        return (self.next() >> 11) * (2.0 ** -53)


@dataclass(frozen=True)
class Gate:
    kind: int
    cycle: int
    q0: int
    q1: int = -1
    theta: float = 0.0
    phi: float = 0.0


@dataclass
class Circuit:
    n: int
    gates: List[Gate]
    rows: int = 0
    cols: int = 0
    depth: int = 0
    seed: int = 0
    param: bool = False
    # indices (into gates) of the parametrised slots, in gate order
    param_gates: List[int] = field(default_factory=list)

    def with_angles(self, thetas, phis) -> "Circuit":
        """Copy with new (theta, phi) on the parametrised slots (for finite
        differences)."""
        gates = list(self.gates)
        for p, gi in enumerate(self.param_gates):
            g = gates[gi]
            gates[gi] = Gate(g.kind, g.cycle, g.q0, g.q1, float(thetas[p]), float(phis[p]))
        return Circuit(self.n, gates, self.rows, self.cols, self.depth, self.seed,
                       self.param, list(self.param_gates))


def cz_patterns(rows: int, cols: int):
    """The 8 CZ layers in rotation order [HZ0, HZ2, VT0, VT2, HZ1, HZ3, VT1, VT3]."""
    def hz(o):
        return [(r * cols + c, r * cols + c + 1)
                for r in range(rows) for c in range(cols - 1)
                if c % 4 == (o + 2 * (r % 2)) % 4]

    def vt(o):
        return [(r * cols + c, (r + 1) * cols + c)
                for r in range(rows - 1) for c in range(cols)
                if r % 4 == (o + 2 * (c % 2)) % 4]

    return [hz(0), hz(2), vt(0), vt(2), hz(1), hz(3), vt(1), vt(3)]


def grid_circuit(rows: int, cols: int, depth: int, seed: int = 0,
                 param: bool = False) -> Circuit:
    """Random grid circuit of ``depth`` cycles (see the module docstring)."""
    if rows < 1 or cols < 1 or depth < 1:
        raise ValueError("rows, cols and depth must be >= 1")
    n = rows * cols
    pats = cz_patterns(rows, cols)
    rng = SplitMix64(seed)
    gates: List[Gate] = [Gate(GATE_H, 0, q) for q in range(n)]
    param_gates: List[int] = []
    had_cz_prev = [False] * n
    had_t = [False] * n
    for t in range(1, depth):
        in_cz = [False] * n
        for a, b in pats[(t - 1) % 8]:
            gates.append(Gate(GATE_CZ, t, a, b))
            in_cz[a] = in_cz[b] = True
        for q in range(n):
            if had_cz_prev[q] and not in_cz[q]:
                if not had_t[q]:
                    had_t[q] = True
                    gates.append(Gate(GATE_T, t, q))
                elif param:
                    theta = math.pi * rng.uniform()
                    phi = 2.0 * math.pi * rng.uniform()
                    param_gates.append(len(gates))
                    gates.append(Gate(GATE_RXY, t, q, -1, theta, phi))
                else:
                    r = rng.next()
                    gates.append(Gate(GATE_X12 if (r >> 63) == 0 else GATE_Y12, t, q))
        had_cz_prev = in_cz
    return Circuit(n, gates, rows, cols, depth, seed, param, param_gates)


def bitstrings(n: int, count: int, seed: int) -> np.ndarray:
    """``count`` uniform n-bit strings with replacement from stream seed+1."""
    if not 1 <= n <= 64:
        raise ValueError("n must be in [1, 64]")
    rng = SplitMix64(seed + 1)
    out = np.empty(count, dtype=np.uint64)
    for i in range(count):
        out[i] = rng.next() >> (64 - n)
    return out


def circuit_from_gates(n: int, gates) -> Circuit:
    """Wrap an explicit gate list (e.g. the paper's App. D example)."""
    gl = [g if isinstance(g, Gate) else Gate(*g) for g in gates]
    pg = [i for i, g in enumerate(gl) if g.kind == GATE_RXY]
    return Circuit(n, gl, param=bool(pg), param_gates=pg)


def gates_as_array(c: Circuit) -> np.ndarray:
    """Structured array view: (kind, cycle, q0, q1, theta, phi) per gate."""
    dt = np.dtype([("kind", np.int32), ("cycle", np.int32), ("q0", np.int32),
                   ("q1", np.int32), ("theta", np.float64), ("phi", np.float64)])
    a = np.empty(len(c.gates), dtype=dt)
    for i, g in enumerate(c.gates):
        a[i] = (g.kind, g.cycle, g.q0, g.q1, g.theta, g.phi)
    return a


# Workloads used across tests and the benchmark: (rows, cols, depth, batch, param)
WORKLOADS = {
    "grid4x4_d10_all": (4, 4, 10, 0, False),
    "grid5x5_d20_b1024": (5, 5, 20, 1024, False),
    "grid6x6_d25_b1000": (6, 6, 25, 1000, False),
    "grid5x9_d40_b1000": (5, 9, 40, 1000, False),
    "grid6x6_d20_b256_param": (6, 6, 20, 256, True),
}

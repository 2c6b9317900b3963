"""Seeded synthetic inputs: the generator's definition and circuit invariants."""
import numpy as np
import pytest

import qgm_inputs as qi


def test_splitmix64_published_vector():
    # Published reference outputs of SplitMix64 for seed 1234567.
    g = qi.SplitMix64(1234567)
    assert [g.next() for _ in range(3)] == [6457827717110365317, 3203168211198807973,
                                          9817491932198370423]


@pytest.mark.parametrize("rows,cols,depth", [(4, 4, 10), (5, 5, 20), (5, 9, 40), (3, 7, 17)])
def test_circuit_rules(rows, cols, depth):
    c = qi.grid_circuit(rows, cols, depth, seed=3)
    n = rows * cols
    assert [g.kind for g in c.gates[:n]] == [qi.GATE_H] * n
    by_cycle = {}
    for g in c.gates:
        by_cycle.setdefault(g.cycle, []).append(g)
    assert max(by_cycle) <= depth - 1
    in_cz = {}
    for t in range(depth):
        used = []
        for g in by_cycle.get(t, []):
            used += [g.q0] if g.q1 < 0 else [g.q0, g.q1]
        assert len(used) == len(set(used)), "a qubit got two gates in one cycle"
        in_cz[t] = {q for g in by_cycle.get(t, []) if g.kind == qi.GATE_CZ for q in (g.q0, g.q1)}
    # every grid edge exactly once per 8 consecutive CZ cycles
    edges = set()
    for r in range(rows):
        for cc in range(cols):
            q = r * cols + cc
            if cc + 1 < cols:
                edges.add((q, q + 1))
            if r + 1 < rows:
                edges.add((q, q + cols))
    if depth >= 9:
        seen = [tuple(sorted((g.q0, g.q1))) for t in range(1, 9) for g in by_cycle[t]
                if g.kind == qi.GATE_CZ]
        assert sorted(seen) == sorted(edges)
    # single-qubit gates: only after a CZ cycle, T first
    had_t = set()
    for t in range(1, depth):
        for g in by_cycle.get(t, []):
            if g.kind == qi.GATE_CZ:
                continue
            assert g.q0 in in_cz[t - 1] and g.q0 not in in_cz[t]
            if g.q0 not in had_t:
                assert g.kind == qi.GATE_T
                had_t.add(g.q0)
            else:
                assert g.kind in (qi.GATE_X12, qi.GATE_Y12)
        for q in range(n):
            if q in in_cz[t - 1] and q not in in_cz[t]:
                assert any(g.q0 == q and g.kind != qi.GATE_CZ for g in by_cycle.get(t, []))


def test_x_y_balance_and_param_mode():
    c = qi.grid_circuit(6, 6, 40, seed=0)
    xy = [g.kind for g in c.gates if g.kind in (qi.GATE_X12, qi.GATE_Y12)]
    frac = xy.count(qi.GATE_X12) / len(xy)
    assert 0.4 < frac < 0.6
    p = qi.grid_circuit(6, 6, 20, seed=0, param=True)
    assert len(p.param_gates) > 0
    th = np.array([p.gates[i].theta for i in p.param_gates])
    ph = np.array([p.gates[i].phi for i in p.param_gates])
    assert th.min() >= 0 and th.max() < np.pi and ph.max() < 2 * np.pi
    # same structure as the fixed-gate circuit: RXY exactly at the X/Y slots
    f = qi.grid_circuit(6, 6, 20, seed=0)
    assert [(g.cycle, g.q0, g.q1) for g in p.gates] == [(g.cycle, g.q0, g.q1) for g in f.gates]
    assert all(f.gates[i].kind in (qi.GATE_X12, qi.GATE_Y12) for i in p.param_gates)


def test_bitstrings_uniform_and_seeded():
    a = qi.bitstrings(25, 4096, seed=0)
    b = qi.bitstrings(25, 4096, seed=0)
    assert (a == b).all() and a.max() < (1 << 25)
    bits = ((a[:, None] >> np.arange(25, dtype=np.uint64)) & np.uint64(1)).astype(float)
    assert np.all(np.abs(bits.mean(0) - 0.5) < 0.05)


def test_seed0_circuits_match_golden():
    # tests/golden/circuits_seed0.json (written by tests/golden/make_golden.py
    # from qgm_inputs): the sha256 of each workload's canonical seed-0 gate
    # list and its gate counts; the C++ generator is checked against this
    # generator gate by gate in tests/test_host_plan.py
    import hashlib
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "circuits_seed0.json")) as f:
        gold = json.load(f)["circuits"]
    assert set(gold) == set(qi.WORKLOADS)
    for name, (rows, cols, depth, _, param) in qi.WORKLOADS.items():
        c = qi.grid_circuit(rows, cols, depth, 0, param=param)
        gl = [(int(g.kind), int(g.cycle), int(g.q0), int(g.q1), f"{float(g.theta):.17g}", f"{float(g.phi):.17g}")
              for g in c.gates]
        assert hashlib.sha256(json.dumps(gl).encode()).hexdigest() == gold[name]["sha256"], name
        assert len(gl) == gold[name]["n_gates"]
        # every qubit starts with H and gets T as its first later one-qubit
        # gate, so H and T each number n
        assert gold[name]["by_kind"]["0"] == rows * cols and gold[name]["by_kind"]["3"] == rows * cols

"""Pins for oracle/order.py (Sec. IV, App. D-E)."""
import itertools
import random

import pytest

import qgm_inputs as qi
from oracle import order as O
from oracle import ugm


def _adj(n, edges):
    a = {i: set() for i in range(n)}
    for u, v in edges:
        a[u].add(v)
        a[v].add(u)
    return a


def test_app_d_graph_and_width(app_d):
    m = ugm.build(app_d)
    full = O.graph(m, open_outputs=True)
    full.update({v: set() for v in m.inputs if v not in full})
    # all six variables: two worldlines of three plus the CZ edge (Eq. ex_ugm)
    g = {v: set() for v in range(6)}
    for f in m.factors:
        if len(f.scope) == 2:
            a, b = f.scope
            g[a].add(b)
            g[b].add(a)
    edges = {tuple(sorted((a, b))) for a in g for b in g[a]}
    assert edges == {(0, 2), (2, 4), (1, 3), (3, 5), (2, 3)}
    # fixing the boundary leaves one edge: width 2 (a 2-clique)
    fixed = O.graph(m)
    assert fixed == {2: {3}, 3: {2}}
    assert O.min_fill(fixed)[1] == 2
    assert O.treewidth_exact(fixed) + 1 == 2


def test_app_e_line_graph_width_4():
    # the line graph printed in App. E (vertices 1..8)
    printed = [(4, 5), (5, 6), (5, 1), (1, 2), (2, 3), (6, 2), (2, 5), (6, 1), (7, 1), (6, 8)]
    a = _adj(9, printed)
    del a[0]
    assert O.treewidth_exact(a) + 1 == 4
    # the line graph of the tensor network drawn for Eq. ex_circ
    tn = [("a", "a2"), ("b", "f"), ("b", "a2"), ("e", "f"), ("b", "c"), ("b", "c2"),
          ("c", "d"), ("c2", "g")]
    lg = O.line_graph(tn)
    assert O.treewidth_exact(lg) + 1 == 4
    assert O.min_fill(lg)[1] == 4


@pytest.mark.parametrize("kind,n,tw", [("path", 9, 1), ("cycle", 8, 2), ("clique", 6, 5),
                                       ("star", 9, 1), ("grid3", 9, 3)])
def test_known_treewidths(kind, n, tw):
    if kind == "path":
        e = [(i, i + 1) for i in range(n - 1)]
    elif kind == "cycle":
        e = [(i, (i + 1) % n) for i in range(n)]
    elif kind == "clique":
        e = list(itertools.combinations(range(n), 2))
    elif kind == "star":
        e = [(0, i) for i in range(1, n)]
    else:
        e = [(r * 3 + c, r * 3 + c + 1) for r in range(3) for c in range(2)] + \
            [(r * 3 + c, r * 3 + c + 3) for r in range(2) for c in range(3)]
    a = _adj(n, e)
    assert O.treewidth_exact(a) == tw
    order, w = O.min_fill(a)
    assert sorted(order) == list(range(n))
    assert w - 1 == tw
    assert O.induced_width(a, order) == w


def test_min_fill_upper_bounds_exact_treewidth():
    rnd = random.Random(11)
    for _ in range(12):
        n = rnd.randint(5, 11)
        e = [p for p in itertools.combinations(range(n), 2) if rnd.random() < 0.35]
        a = _adj(n, e)
        order, w = O.min_fill(a)
        assert w - 1 >= O.treewidth_exact(a)
        assert O.induced_width(a, order) == w


def test_min_fill_tie_break_on_a_chain():
    # all chain ends have fill 0 and degree 1: the smallest id goes first
    a = _adj(5, [(0, 1), (1, 2), (2, 3), (3, 4)])
    assert O.min_fill(a)[0] == [0, 1, 2, 3, 4]
    a = _adj(5, [(4, 3), (3, 1), (1, 2), (2, 0)])
    assert O.min_fill(a)[0][0] == 0


def test_vertical_order_is_lexicographic():
    c = qi.grid_circuit(2, 3, 10, 0)
    m = ugm.build(c)
    vs = list(range(m.n_vars))
    order = O.vertical(m, vs, 2, 3)           # rows < cols: j runs down columns
    rank = O.qubit_rank(2, 3)
    assert rank == [0, 2, 4, 1, 3, 5]
    keys = [(rank[m.var_qubit[v]], m.var_k[v]) for v in order]
    assert keys == sorted(keys)
    assert O.qubit_rank(3, 3) == list(range(9))


def test_app_d_tensor_network_line_graph_width_4(app_d):
    # App. E: the App. D circuit as a tensor network; its line graph is the
    # 4-clique of the CZ's segments (width 4, against 2 for the graphical model)
    tn = O.tensor_network(app_d)
    assert tn == [(0, 2), (1, 2), (2, 3), (2, 4)]
    lg = O.line_graph(tn)
    assert O.treewidth_exact(lg) + 1 == 4
    assert O.min_fill(lg)[1] == 4


def test_tensor_network_segments_and_chain():
    # one qubit, k gates: k - 1 segments, a path (width 2); segment count is
    # the sum over qubits of (gates on the qubit - 1)
    G = qi.Gate
    chain = qi.circuit_from_gates(1, [G(qi.GATE_H, t, 0) for t in range(6)])
    lg = O.line_graph(O.tensor_network(chain))
    assert len(lg) == 5 and O.treewidth_exact(lg) + 1 == 2
    c = qi.grid_circuit(3, 3, 9, 1)
    per_q = [sum(1 for g in c.gates if q in (g.q0, g.q1)) for q in range(c.n)]
    assert len(O.tensor_network(c)) == sum(k - 1 for k in per_q)


@pytest.mark.parametrize("rows,cols,depth,seed", [(2, 2, 6, 0), (2, 3, 5, 1), (1, 4, 8, 2)])
def test_graphical_model_never_wider_than_line_graph(rows, cols, depth, seed):
    # the interaction graph is a minor of the line graph (segments joined by
    # diagonal gates are one variable), so its treewidth is never larger
    c = qi.grid_circuit(rows, cols, depth, seed)
    ugm_g = O.graph(ugm.build(c))
    lg = O.line_graph(O.tensor_network(c))
    if len(lg) > 18:
        pytest.skip("exact treewidth too slow")
    assert O.treewidth_exact(ugm_g) <= O.treewidth_exact(lg)

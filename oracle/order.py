"""Elimination orders and widths (oracle; test only).

Sec. IV.B of the paper: eliminating a vertex joins all of its neighbours;
the cliques made this way are the factors variable elimination creates; the
size of the largest one is the induced width of the order (the paper's
example calls a 2-vertex clique "treewidth 2", Fig. 4 plots size - 1).
Functions here report ``max_clique`` (size convention) and leave ``- 1`` to
the caller.

* ``graph``: the interaction graph G of Sec. III.B on the free variables --
  one vertex per variable not fixed by a boundary delta, a clique per factor.
* ``min_fill``: greedy order, each step the vertex whose elimination adds the
  fewest fill edges; ties by fewest neighbours, then smallest id (the paper
  used QuickBB, which is third-party; min-fill is the library's heuristic).
* ``vertical``: Sec. IV.A -- worldline after worldline, lexicographic (j, k),
  qubits numbered along the smaller lateral dimension first.
* ``treewidth_exact``: subset dynamic programme TW(S) = min_v max(TW(S-v),
  |Q(S-v, v)|) (Bodlaender, Fomin, Koster, Kratsch, Thilikos 2006); small
  graphs only, used to pin the heuristics from below.
* ``cliques`` and ``slice_greedy``: the cliques an order makes, and slicing
  (conditioning on variables, Sec. IV's remark that fixing a variable splits
  the sum into independent parts) chosen greedily: repeatedly fix the
  variable that lies in the most cliques of the largest size (ties: smallest
  id), removing it from the graph before the cliques are recounted.
* ``line_graph``: App. E's construction.
* ``tensor_network``: App. E's tensor network of a circuit, one tensor per
  gate, as its wire segments between two gates (the segments to the fixed
  input and output vectors are fixed indices and drop out, as the boundary
  variables do in ``graph``).
Parity: pinned (App. D example width 2, App. E line graph width 4 -- from the
printed graph and from the App. D circuit's tensor network --, chains,
cycles, trees and cliques against their known treewidths, exact DP as a lower
bound, the interaction graph a minor of the line graph so never wider;
tests/test_oracle_order.py).
"""
from itertools import combinations


def graph(model, open_outputs=False):
    fixed = set(model.inputs)
    if not open_outputs:
        fixed |= set(model.outputs)
    verts = [v for v in range(model.n_vars) if v not in fixed]
    adj = {v: set() for v in verts}
    for f in model.factors:
        s = [v for v in f.scope if v not in fixed]
        for a, b in combinations(s, 2):
            if a != b:
                adj[a].add(b)
                adj[b].add(a)
    return adj


def _copy(adj):
    return {v: set(n) for v, n in adj.items()}


def _eliminate(adj, v):
    nb = adj.pop(v)
    for a in nb:
        adj[a].discard(v)
        adj[a] |= nb - {a}
    return nb


def induced_width(adj, order):
    """Max clique size (vertex + its remaining neighbours) along ``order``."""
    g = _copy(adj)
    w = 0
    for v in order:
        w = max(w, 1 + len(g[v]))
        _eliminate(g, v)
    return w


def min_fill(adj, keep=()):
    """Min-fill order of all vertices not in ``keep``; returns (order, max_clique)."""
    g = _copy(adj)
    keep = set(keep)
    order = []
    w = 0
    while len(g) > len(keep):
        best = None
        for v in sorted(g):
            if v in keep:
                continue
            nb = sorted(g[v])
            fill = 0
            for i in range(len(nb)):
                for j in range(i + 1, len(nb)):
                    if nb[j] not in g[nb[i]]:
                        fill += 1
            key = (fill, len(nb), v)
            if best is None or key < best:
                best = key
        v = best[2]
        w = max(w, 1 + len(g[v]))
        _eliminate(g, v)
        order.append(v)
    return order, w


def cliques(adj, order, removed=()):
    """Cliques (vertex + remaining neighbours) along ``order`` on the graph
    without the vertices in ``removed``; vertices of ``removed`` are skipped."""
    removed = set(removed)
    g = {v: set(n) - removed for v, n in adj.items() if v not in removed}
    out = []
    for v in order:
        if v in removed:
            continue
        out.append({v} | g[v])
        _eliminate(g, v)
    return out


def slice_greedy(adj, order, n_slices=None, max_clique=None, allowed=None):
    """Greedy slicing: fix, one at a time, the variable (from ``allowed``,
    default the vertices of ``order``) in the most cliques of the largest
    size along ``order``, ties to the smallest id; stop after ``n_slices``
    variables or once the largest clique is at most ``max_clique``."""
    allowed = set(order if allowed is None else allowed)
    chosen = []
    while True:
        cl = cliques(adj, order, chosen)
        mx = max((len(c) for c in cl), default=0)
        if n_slices is not None and len(chosen) >= n_slices:
            break
        if max_clique is not None and mx <= max_clique:
            break
        count = {}
        for c in cl:
            if len(c) == mx:
                for v in c:
                    if v in allowed:
                        count[v] = count.get(v, 0) + 1
        if not count:
            break
        chosen.append(min(count, key=lambda v: (-count[v], v)))
    return chosen


def qubit_rank(rows, cols, transpose=False):
    """Qubit numbering j of Sec. IV.A: neighbours along the smaller lateral
    dimension get consecutive j (ties: along a row)."""
    colmajor = rows < cols
    if transpose:
        colmajor = not colmajor
    n = rows * cols
    rank = [0] * n
    for q in range(n):
        r, c = divmod(q, cols)
        rank[q] = c * rows + r if colmajor else q
    return rank


def vertical(model, verts, rows, cols, transpose=False):
    """Vertices of ``verts`` in lexicographic (j, k) order."""
    rank = qubit_rank(rows, cols, transpose)
    return sorted(verts, key=lambda v: (rank[model.var_qubit[v]], model.var_k[v], v))


def treewidth_exact(adj):
    """Exact treewidth (max bag size - 1) by the subset recursion; <= ~14 vertices."""
    verts = sorted(adj)
    n = len(verts)
    if n == 0:
        return -1
    ix = {v: i for i, v in enumerate(verts)}
    nbm = [0] * n
    for v in verts:
        for u in adj[v]:
            nbm[ix[v]] |= 1 << ix[u]

    def q_size(S, i):
        # vertices outside S + {i} reachable from i through S
        seen = 1 << i
        frontier = 1 << i
        reach = 0
        while frontier:
            nxt = 0
            f = frontier
            while f:
                b = f & -f
                f ^= b
                nxt |= nbm[b.bit_length() - 1]
            nxt &= ~seen
            seen |= nxt
            reach |= nxt & ~S
            frontier = nxt & S
        return bin(reach & ~(1 << i)).count("1")

    full = (1 << n) - 1
    TW = {0: -1}
    for size in range(1, n + 1):
        for comb in combinations(range(n), size):
            S = 0
            for i in comb:
                S |= 1 << i
            best = n
            for i in comb:
                rest = S & ~(1 << i)
                best = min(best, max(TW[rest], q_size(rest, i)))
            TW[S] = best
    return TW[full]


def line_graph(edges):
    """App. E: one vertex per edge of G, adjacent when the edges share a vertex."""
    adj = {i: set() for i in range(len(edges))}
    for i, j in combinations(range(len(edges)), 2):
        if set(edges[i]) & set(edges[j]):
            adj[i].add(j)
            adj[j].add(i)
    return adj


def tensor_network(circuit):
    """Wire segments between two gates as (producer, consumer) gate indices,
    in the order their consumers close them (gate order, first qubit first)."""
    last = {}
    edges = []
    for gi, g in enumerate(circuit.gates):
        for q in ([g.q0] if g.q1 < 0 else [g.q0, g.q1]):
            if q in last:
                edges.append((last[q], gi))
            last[q] = gi
    return edges

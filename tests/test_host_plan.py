"""Host side of the C ABI (no GPU): circuit generator, model and planner
against the oracle, bit-exact, plus error paths and the exported symbols."""
import ctypes
import os
import re

import numpy as np
import pytest

import qgm_inputs as qi
from oracle import order as O
from oracle import ugm

Q = pytest.importorskip("paper_1712_05384_gb300")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1712_05384_gb300 import build
    build.build()


def test_every_declared_symbol_is_exported():
    hdr = open(os.path.join(ROOT, "include", "qgm.h")).read()
    names = sorted(set(re.findall(r"\b(qgm_[a-z0-9_]+)\s*\(", hdr)))
    assert len(names) >= 20
    L = ctypes.CDLL(Q._lib.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("rows,cols,depth,param", [(4, 4, 10, False), (5, 5, 20, False),
                                                   (5, 9, 40, False), (6, 6, 20, True),
                                                   (3, 7, 13, True)])
def test_generator_bit_exact(rows, cols, depth, param):
    py = qi.grid_circuit(rows, cols, depth, 0, param=param)
    cc = Q.Circuit.grid(rows, cols, depth, 0, param)
    assert cc.gates() == [(g.kind, g.cycle, g.q0, g.q1, g.theta, g.phi) for g in py.gates]
    assert list(cc.param_gates()) == py.param_gates


@pytest.mark.parametrize("rows,cols,depth", [(4, 4, 10), (6, 6, 25)])
def test_model_matches_oracle(rows, cols, depth):
    py = qi.grid_circuit(rows, cols, depth, 0)
    m = Q.Model(Q.Circuit.grid(rows, cols, depth, 0))
    om = ugm.build(py)
    q, k = m.vars()
    assert list(q) == om.var_qubit and list(k) == om.var_k
    assert m.info.n_vars == om.n_vars and m.info.n_nondiag == om.n_nondiag
    assert m.factors() == [tuple(f.scope) for f in om.factors]
    # diagonal gates add no variable (Sec. III.A): n_vars = n + #non-diagonal
    nd = sum(g.kind in (qi.GATE_H, qi.GATE_X12, qi.GATE_Y12, qi.GATE_RXY) for g in py.gates)
    assert m.info.n_vars == py.n + nd


@pytest.mark.parametrize("rows,cols,depth,mode", [(4, 4, 10, 1), (4, 4, 14, 0), (5, 5, 20, 0),
                                                  (3, 6, 16, 1), (5, 6, 16, 0)])
def test_min_fill_order_bit_exact(rows, cols, depth, mode):
    py = qi.grid_circuit(rows, cols, depth, 0)
    om = ugm.build(py)
    m = Q.Model(Q.Circuit.grid(rows, cols, depth, 0))
    p = Q.Plan(m, order_kind=Q.ORDER_MINFILL, output_mode=mode, batch=16)
    adj = O.graph(om, open_outputs=(mode == 1))
    keep = set(om.outputs) if mode == 1 else set()
    oo, w = O.min_fill(adj, keep)
    assert list(p.order()) == oo
    assert p.info.max_clique == w
    assert O.induced_width(adj, oo) == w


@pytest.mark.parametrize("rows,cols,depth", [(4, 4, 10), (5, 9, 12), (6, 4, 14)])
def test_vertical_orders_bit_exact(rows, cols, depth):
    py = qi.grid_circuit(rows, cols, depth, 0)
    om = ugm.build(py)
    m = Q.Model(Q.Circuit.grid(rows, cols, depth, 0))
    adj = O.graph(om)
    for kind, tr in ((Q.ORDER_VERTICAL, False), (Q.ORDER_VERTICAL_T, True)):
        p = Q.Plan(m, order_kind=kind, batch=4)
        ref = O.vertical(om, sorted(adj), rows, cols, transpose=tr)
        assert list(p.order()) == ref
        assert p.info.max_clique == O.induced_width(adj, ref)


def test_auto_picks_cheapest():
    m = Q.Model(Q.Circuit.grid(5, 5, 20, 0))
    costs = {}
    for kind in (Q.ORDER_MINFILL, Q.ORDER_VERTICAL, Q.ORDER_VERTICAL_T):
        p = Q.Plan(m, order_kind=kind, batch=64)
        costs[kind] = p.info.bytes_per_slice * p.info.n_slices
    auto = Q.Plan(m, order_kind=Q.ORDER_AUTO, batch=64)
    assert auto.info.bytes_per_slice * auto.info.n_slices == min(costs.values())


def test_given_order_and_validation():
    py = qi.grid_circuit(3, 3, 10, 0)
    om = ugm.build(py)
    m = Q.Model(Q.Circuit.grid(3, 3, 10, 0))
    adj = O.graph(om)
    order = sorted(adj, reverse=True)
    p = Q.Plan(m, order=order, batch=8)
    assert list(p.order()) == order
    assert p.info.max_clique == O.induced_width(adj, order)
    with pytest.raises(Q.QgmError):
        Q.Plan(m, order=order[:-1], batch=8)          # missing variable
    with pytest.raises(Q.QgmError):
        Q.Plan(m, order=order + [order[0]], batch=8)  # repeated variable
    with pytest.raises(Q.QgmError):
        Q.Plan(m, batch=0)
    with pytest.raises(Q.QgmError):
        Q.Plan(m, output_mode=7)


def test_slicing_respects_budget():
    m = Q.Model(Q.Circuit.grid(5, 5, 20, 0))
    full = Q.Plan(m, order_kind=Q.ORDER_MINFILL, batch=64)
    budget = full.info.arena_bytes // 6
    p = Q.Plan(m, order_kind=Q.ORDER_MINFILL, batch=64, mem_budget_bytes=budget)
    assert p.info.n_slices > 1 and p.info.arena_bytes <= budget
    sv = p.slice_vars()
    assert len(sv) == p.info.n_slice_vars and len(set(sv)) == len(sv)
    # sliced variables are free variables of the order (they are skipped
    # there), and slicing narrows the order's cliques
    assert set(sv) <= set(p.order()) and p.info.n_free == len(p.order())
    assert p.info.max_clique < full.info.max_clique
    with pytest.raises(Q.QgmError):
        Q.Plan(m, order_kind=Q.ORDER_MINFILL, batch=64, mem_budget_bytes=1024)


def test_steps_are_consistent():
    m = Q.Model(Q.Circuit.grid(4, 4, 12, 0))
    p = Q.Plan(m, batch=8)
    st = p.steps()
    assert (st["n_in"] >= 1).all() and (st["n_in"] <= 8).all()
    assert (st["k"] >= 0).all() and st["k"].sum() == p.info.n_free
    assert st["out_rank"][-1] == 0 and st["batched"][-1] == 1


def test_partially_open_outputs_plan():
    # Eq. psi_x with the deltas of k chosen outputs omitted: those variables
    # are never eliminated and the final tensor keeps them (k axes) beside
    # the batch axis
    m = Q.Model(Q.Circuit.grid(4, 4, 12, 0))
    closed = Q.Plan(m, batch=8)
    mask = (1 << 1) | (1 << 6) | (1 << 13)
    p = Q.Plan(m, batch=8, open_mask=mask)
    assert p.n_open == 3
    st = p.steps()
    # output variables are fixed by the bitstring or open: neither is eliminated
    assert st["k"].sum() == p.info.n_free == closed.info.n_free
    assert st["out_rank"][-1] == 3 and st["batched"][-1] == 1
    with pytest.raises(Q.QgmError):
        Q.Plan(m, batch=8, open_mask=1 << 16)          # no qubit 16 on a 4x4 grid
    with pytest.raises(Q.QgmError):
        Q.Plan(m, batch=8, open_mask=mask, gradients=True)


def test_contraction_trees_need_fewer_products():
    # 5x5 depth 20: buckets of three or more large inputs multiplied pairwise
    # (each variable summed once no other factor holds it) need well under
    # the products of the single product-sum per bucket; same variables
    m = Q.Model(Q.Circuit.grid(5, 5, 20, 0))
    plain = Q.Plan(m, batch=64)
    tree = Q.Plan(m, batch=64, trees=True)
    assert tree.info.n_free == plain.info.n_free
    assert tree.info.max_clique == plain.info.max_clique
    f_plain, f_tree = plain.step_costs()[1].sum(), tree.step_costs()[1].sum()
    assert f_tree < 0.8 * f_plain
    st = tree.steps()
    assert st["k"].sum() == tree.info.n_free


@pytest.mark.parametrize("rows,cols,depth,B,n_gemm,n_tc,n_fp32", [(4, 5, 30, 16, 1, 1, 1), (4, 6, 34, 6, 5, 4, 3),
                                                                (4, 8, 40, 4, 4, 4, 3)])
def test_tensor_core_gemm_steps(rows, cols, depth, B, n_gemm, n_tc, n_fp32):
    # GEMM steps (min-fill) and their (m, n, k, s) variable counts with both
    # operands' batch flags.  For the FP32-core kernel a step needs >= 6
    # private variables on one side, >= 6 (>= 5 with 64 or more batch
    # entries) on the other and k >= 4: 4x6 d34 has (8, 6, 8), (9, 6, 4),
    # (6, 6, 8); 4x8 d40 (8, 8, 8), (11, 7, 8), (11, 9, 8).  On the tensor
    # cores a step needs an M side of >= 128 rows (batch entries count as
    # rows when the other operand has no batch axis: 4x6 d34's batch of 6
    # pads to 8), an N side of >= 32 and, below 16 summed entries, an output
    # of >= 2^20 entries (the chunk is zero-padded): 4x6 d34 gains (7, 7, 2)
    # and (11, 5, 2) and loses (6, 6, 8) (2^6 rows, both batched); 4x8 d40
    # gains (10, 9, 2)
    m = Q.Model(Q.Circuit.grid(rows, cols, depth, 0))
    p = Q.Plan(m, order_kind=1, batch=B)
    assert (p.info.n_gemm_steps, p.info.n_gemm_tc_steps) == (n_gemm, n_tc)
    assert Q.Plan(m, order_kind=1, batch=B, precision="bf16").info.n_gemm_tc_steps == n_tc
    off = Q.Plan(m, order_kind=1, batch=B, precision="fp32")
    assert (off.info.n_gemm_steps, off.info.n_gemm_tc_steps) == (n_fp32, 0)
    assert Q.Plan(m, order_kind=1, batch=B, gemm=False).info.n_gemm_tc_steps == 0


def test_nested_steps_keep_the_product_sum():
    # 5x5 depth 20: the two widest buckets sum part of their variables in an
    # inner loop over the inputs that alone hold them; the steps still list
    # every summed variable once (the other executors run them flat)
    m = Q.Model(Q.Circuit.grid(5, 5, 20, 0))
    p = Q.Plan(m, batch=1024)
    assert p.info.n_nested_steps >= 2
    st = p.steps()
    assert st["k"].sum() == p.info.n_free


@pytest.mark.parametrize("rows,cols,depth,seed", [(3, 3, 8, 0), (4, 4, 12, 1), (3, 5, 16, 2),
                                                  (2, 6, 10, 3)])
def test_line_graph_width_bit_exact(rows, cols, depth, seed):
    # App. E (ordering study, Fig. 6): the planner's line graph of the
    # circuit's tensor network and its min-fill width equal the oracle's
    c = qi.grid_circuit(rows, cols, depth, seed)
    edges = O.tensor_network(c)
    ref = O.min_fill(O.line_graph(edges))[1]
    ns, w = Q.Circuit.grid(rows, cols, depth, seed).line_graph_width()
    assert ns == len(edges) and w == ref


def test_line_graph_width_app_d(app_d):
    c = Q.Circuit.from_gates(2, app_d.gates)
    assert c.line_graph_width() == (4, 4)


def test_ordering_study_rows():
    from paper_1712_05384_gb300 import study
    r = study.widths(4, 4, 12)
    m = Q.Model(Q.Circuit.grid(4, 4, 12, 0))
    assert r["min_fill"] == Q.Plan(m, order_kind=Q.ORDER_MINFILL).info.max_clique - 1
    assert r["line_graph"] + 1 == Q.Circuit.grid(4, 4, 12, 0).line_graph_width()[1]
    assert r["line_graph"] >= r["min_fill"]


@pytest.mark.parametrize("rows,cols,depth,seed,pauli", [(2, 3, 6, 0, "IZIIII"), (3, 3, 5, 1, "XIIIYIIIZ"),
                                                        (2, 2, 8, 2, "YYXZ"), (3, 3, 3, 3, "IIIIXIIII"),
                                                        (2, 3, 4, 4, "ZIIIIX")])
def test_observable_circuit_reproduces_expectation(rows, cols, depth, seed, pauli):
    # Sec. III: <0|U^dagger P U|0> = phase * <0|W|0> with W built on the host
    # from the light cone; W's amplitude by the oracle's state vector, the
    # expectation by the oracle's definition
    from oracle import observable as OB
    from oracle import statevector as sv
    c = qi.grid_circuit(rows, cols, depth, seed)
    w, phase, qmap = Q.Circuit.grid(rows, cols, depth, seed).observable(pauli)
    keep, support = OB.light_cone(c, pauli)
    assert sorted(np.nonzero(qmap >= 0)[0].tolist()) == support
    gates = [qi.Gate(*g) for g in w.gates()]
    # the light-cone gates come first, renumbered
    for g, gi in zip(gates, keep):
        o = c.gates[gi]
        assert (g.kind, g.q0) == (o.kind, int(qmap[o.q0]))
    wc = qi.circuit_from_gates(len(support), gates)
    assert abs(phase * sv.state(wc)[0] - OB.expectation(c, pauli)) < 1e-12
    assert Q.Circuit.grid(rows, cols, depth, seed).observable("I" * c.n)[0] is None
    with pytest.raises(Q.QgmError):
        Q.Circuit.grid(rows, cols, depth, seed).observable("Q" * c.n)


@pytest.mark.parametrize("rows,cols,depth,batch,div", [
    (5, 5, 20, 64, 3), (5, 5, 20, 64, 20), (6, 6, 25, 8, 4), (4, 5, 30, 16, 10), (5, 9, 40, 1, 64)])
def test_slicer_bit_exact(rows, cols, depth, batch, div):
    # Slicing conditions on variables (Sec. IV); the choice is the greedy
    # rule restated independently in oracle.order.slice_greedy: the variable
    # in the most largest-size cliques along the order, ties to the smallest
    # id.  The library stops when its live set fits the budget; the oracle is
    # asked for the same number of variables and must pick the same ones.
    m = Q.Model(Q.Circuit.grid(rows, cols, depth, 0))
    full = Q.Plan(m, order_kind=Q.ORDER_MINFILL, batch=batch)
    p = Q.Plan(m, order_kind=Q.ORDER_MINFILL, batch=batch, mem_budget_bytes=full.info.arena_bytes // div)
    sv = [int(v) for v in p.slice_vars()]
    assert len(sv) >= 1
    om = ugm.build(qi.grid_circuit(rows, cols, depth, 0))
    adj = O.graph(om)
    order = [int(v) for v in p.order()]
    assert O.slice_greedy(adj, order, n_slices=len(sv)) == sv
    # the reported width is the order's largest clique without those variables
    assert p.info.max_clique == max(len(c) for c in O.cliques(adj, order, sv))


@pytest.mark.parametrize("rows,cols,depth,batch", [(5, 9, 40, 4), (6, 6, 25, 1000), (4, 8, 40, 4), (6, 6, 25, 1),
                                                   (7, 7, 20, 1)])
def test_gemm_shapes_fit_the_launch(rows, cols, depth, batch):
    # a GEMM-shaped step launches one set of tiles per shared kept index:
    # at most 2^15 of them, and every variable class fits the descriptor
    p = Q.Plan(Q.Model(Q.Circuit.grid(rows, cols, depth, 0)), batch=batch, executor=Q.EXEC_STEPWISE)
    gs = p.gemm_shapes()
    assert len(gs) == p.info.n_gemm_steps
    kinds = p.step_kernels()
    for g in gs:
        assert kinds[g["step"]] == 3
        assert g["ns"] <= 15 and max(g["nm"], g["nn"], g["nk"]) < 24
        if g["tc"]:
            assert g["nk"] >= 2 and min(g["nm"], g["nn"]) >= 5
        else:
            assert g["nk"] >= 4 and max(g["nm"], g["nn"]) >= 6 and min(g["nm"], g["nn"]) >= 5
    assert sum(g["tc"] for g in gs) == p.info.n_gemm_tc_steps


@pytest.mark.parametrize("rows,cols,depth,batch,kw", [(5, 9, 40, 4, {"gemm": False, "trees": True}),
                                                     (5, 9, 40, 4, {"trees": True}), (4, 8, 40, 4, {"trees": True}),
                                                     (6, 6, 25, 1000, {"trees": True}), (5, 5, 20, 64, {"trees": True})])
def test_contraction_trees_keep_every_tensor(rows, cols, depth, batch, kw):
    # App. A bucket elimination is a tree: every intermediate feeds exactly
    # one step (the planner refuses a plan that breaks this).  A bucket's
    # contraction tree must sum a variable held by a single input at that
    # input's parent: 5x9 depth 40 with trees has such buckets; each summed
    # variable must disappear exactly once (sum of k = eliminated variables)
    m = Q.Model(Q.Circuit.grid(rows, cols, depth, 0))
    p = Q.Plan(m, order_kind=1, batch=batch, executor=Q.EXEC_STEPWISE, **kw)
    st = p.steps()
    assert st["k"].sum() == p.info.n_free
    assert st["out_rank"][-1] == 0


def test_set_params_checks_its_arguments():
    # new angles keep the plan's structure; the count must match 2 per RXY gate
    c = Q.Circuit.grid(3, 3, 10, 1, True)
    p = Q.Plan(Q.Model(c), batch=4, gradients=True)
    n = 2 * len(c.param_gates())
    p.set_params(np.linspace(0.1, 3.0, n))
    with pytest.raises(Q.QgmError):
        p.set_params(np.zeros(n + 2))
    # a sliced gradient plan is accepted (each slice recomputed in turn)
    m = Q.Model(Q.Circuit.grid(4, 5, 20, 2, True))
    full = Q.Plan(m, batch=8, gradients=True, executor=Q.EXEC_STEPWISE)
    s = Q.Plan(m, batch=8, gradients=True, executor=Q.EXEC_STEPWISE, mem_budget_bytes=full.info.arena_bytes // 3)
    assert s.info.n_slices > 1


def test_torch_complex_gradient_convention():
    # the autograd wrapper relies on torch passing G = 2 dL/d(conj a) for a
    # complex output and expecting dL/dp = Re sum conj(G) da/dp: for
    # L = |a|^2 with a = (1 + 2i) p at p = 1, dL/dp = 2 |1 + 2i|^2 = 10
    torch = pytest.importorskip("torch")
    p = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    z = torch.tensor(1 + 2j, dtype=torch.complex128, requires_grad=True)
    (z * z.conj()).real.backward()
    assert complex(z.grad) == 2 * (1 + 2j)        # G = 2 dL/dconj(z) = 2 z
    a = (1 + 2j) * p.to(torch.complex128)
    (a * a.conj()).real.backward()
    assert abs(p.grad.item() - 10.0) < 1e-12


def test_batch_outer_intermediates():
    # a product per batch entry on the tensor cores whose output only another
    # tensor-core step reads keeps the batch entry outermost: on 5x9 depth 40
    # (4 bitstrings) the two large per-entry products feed folded GEMMs
    m = Q.Model(Q.Circuit.grid(5, 9, 40, 0))
    gs = Q.Plan(m, order_kind=1, batch=4, executor=Q.EXEC_STEPWISE).gemm_shapes()
    prod = [g for g in gs if g["o_bout"]]
    cons = [g for g in gs if g["in_bout"]]
    assert len(prod) == len(cons) == 2
    for g in prod:
        assert g["tc"] and g["a_bat"] and g["b_bat"]
    # never with the FP32-core GEMM (no tensor-core steps) or a gradient layout
    for kw in ({"precision": "fp32"}, {"gradients": True, "batch": 2}):
        kw = dict({"batch": 4}, **kw)
        p = Q.Plan(Q.Model(Q.Circuit.grid(4, 6, 30, 0)), order_kind=1, executor=Q.EXEC_STEPWISE, **kw)
        assert not any(g["o_bout"] or g["in_bout"] for g in p.gemm_shapes())


def test_small_batch_free_steps_run_in_groups():
    # runs of two or more consecutive small steps without a batch axis (at
    # most 2^12 outputs and 2^16 products) share one single-CTA launch
    # (kind 4); every grouped step is such a step, and such a step outside a
    # group has a non-small or batched neighbour on both sides
    p = Q.Plan(Q.Model(Q.Circuit.grid(5, 9, 40, 0)), batch=4, order_kind=Q.ORDER_MINFILL,
               executor=Q.EXEC_STEPWISE)
    kinds = p.step_kernels()
    st = p.steps()
    small = (st["batched"] == 0) & (st["out_rank"] <= 12) & (st["out_rank"] + st["k"] <= 16) & (kinds != 3)
    assert (kinds == 4).sum() > 100
    assert np.all(small[kinds == 4])
    for s in np.nonzero(small & (kinds != 4))[0]:
        assert not (s > 0 and small[s - 1]) and not (s + 1 < len(kinds) and small[s + 1])


@pytest.mark.parametrize("rows,cols,depth,batch", [(5, 9, 40, 4), (4, 8, 40, 16), (4, 6, 34, 6)])
def test_folded_steps_are_the_convertible_ones(rows, cols, depth, batch):
    # a tensor-core step can convert its streamed operand in the product
    # kernel exactly when its batch entries fold into M: the output and one
    # operand carry the batch axis, the other does not (and the batch has
    # more than one entry)
    p = Q.Plan(Q.Model(Q.Circuit.grid(rows, cols, depth, 0)), batch=batch, order_kind=Q.ORDER_MINFILL,
               executor=Q.EXEC_STEPWISE)
    gs = p.gemm_shapes()
    assert any(g["conv_ok"] for g in gs)
    for g in gs:
        fold = g["tc"] and g["o_bat"] and (g["a_bat"] != g["b_bat"]) and batch > 1
        assert g["conv_ok"] == int(bool(fold)), g

"""Adjoint elimination (qgm_amplitude_grad) against the FP64 oracle (GPU).

Tolerance (gradients): per component |g - g_ref| <= 1e-3 max(|g_ref|,
1e-2 max_j |g_ref,j|) -- relative 1e-3 with a floor for components that
nearly vanish; the reference is the oracle's derivative-insertion gradient,
itself pinned against central finite differences.
"""
import numpy as np
import pytest

import qgm_inputs as qi
from oracle import grad as OG
from oracle import statevector as sv
from oracle import ve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    from paper_1712_05384_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1712_05384_gb300 as q
    q.lib()
    return q


def close(g, ref):
    floor = 1e-2 * np.max(np.abs(ref))
    return np.all(np.abs(g - ref) <= 1e-3 * np.maximum(np.abs(ref), floor)), \
        np.max(np.abs(g - ref) / np.maximum(np.abs(ref), floor))


def gpu_grad(q, c, bits, weights=None):
    plan = q.Plan(q.Model(q.Circuit.grid(c.rows, c.cols, c.depth, c.seed, True)),
                  batch=len(bits), gradients=True).bind()
    B = len(bits)
    d_bits = torch.from_numpy(bits.astype(np.int64)).cuda()
    if weights is None:
        a = sv.amplitudes(c, bits)
        weights = a / np.abs(a) ** 2
    w = np.zeros(2 * B)
    w[0::2], w[1::2] = weights.real, weights.imag
    d_w = torch.from_numpy(w).cuda()
    n_par = 2 * len(c.param_gates)
    d_grad = torch.zeros(n_par, dtype=torch.float64, device="cuda")
    d_amp = torch.zeros(2 * B, dtype=torch.float64, device="cuda")
    plan.amplitude_grad(d_bits, d_w, d_grad, d_amp)
    torch.cuda.synchronize()
    assert plan.status() == 0
    o = d_amp.cpu().numpy()
    return d_grad.cpu().numpy(), o[0::2] + 1j * o[1::2]


@pytest.mark.parametrize("rows,cols,depth,seed,B", [(3, 3, 12, 4, 16), (2, 4, 16, 1, 7),
                                                    (3, 4, 10, 2, 33)])
def test_gradient_small_vs_oracle(q, rows, cols, depth, seed, B):
    c = qi.grid_circuit(rows, cols, depth, seed, param=True)
    bits = qi.bitstrings(c.n, B, seed)
    g, a = gpu_grad(q, c, bits)
    ref = OG.grad_exact(c, bits)
    ok, worst = close(g, ref)
    assert ok, worst
    assert np.max(np.abs(a - sv.amplitudes(c, bits))) * 2 ** (c.n / 2) < 1e-5


def test_gradient_matches_finite_differences(q):
    c = qi.grid_circuit(3, 3, 12, 6, param=True)
    bits = qi.bitstrings(c.n, 10, 6)
    g, _ = gpu_grad(q, c, bits)
    fd = OG.grad_fd(c, bits, h=1e-4)
    ref = np.array([fd[i] for i in range(len(g))])
    ok, worst = close(g, ref)
    assert ok, worst


def test_grid6x6_d20_b256_full_loss_vs_oracle(q):
    # 6x6 grid, depth 20, parametrised angles, all 256 bitstrings: the
    # gradient of L = sum_x log |a_x|^2 (App. B's log-probability loss)
    # through the torch.autograd wrapper, against the oracle's gradient for 48
    # of the 362 angles (tests/golden/grad_grid6x6_d20.json: derivative
    # insertion with the plain-C elimination)
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "grad_grid6x6_d20.json")) as f:
        gold = json.load(f)
    c = qi.grid_circuit(6, 6, 20, 0, param=True)
    bits = qi.bitstrings(c.n, 256, 0)
    plan = q.Plan(q.Model(q.Circuit.grid(6, 6, 20, 0, True)), batch=256, gradients=True).bind()
    th, ph = OG.params(c)
    params = torch.tensor(np.stack([th, ph], axis=1).reshape(-1), dtype=torch.float64, requires_grad=True)
    assert params.numel() == gold["n_params"]
    d_bits = torch.from_numpy(bits.astype(np.int64)).cuda()
    a = q.autograd.amplitudes(plan, params, d_bits)
    L = torch.sum(torch.log(torch.abs(a) ** 2))
    assert abs(L.item() - gold["sum_log_p"]) < 1e-4 * abs(gold["sum_log_p"])
    L.backward()
    assert plan.status() == 0
    g = params.grad.numpy()
    idx = [e["param"] for e in gold["grad"]]
    ref = np.array([e["dL"] for e in gold["grad"]])
    ok, worst = close(g[idx], ref)
    print(f"[grad] 6x6 d20, 256 bitstrings, {len(idx)} angles: worst scaled error {worst:.2e}")
    assert ok, worst


def test_autograd_small_and_new_angles(q):
    # the autograd wrapper on 3x3 depth 12: L = sum log|a|^2 against the
    # oracle's derivative insertion; then new angles through the same plan
    # (qgm_plan_set_params, no re-planning) give the other circuit's
    # amplitudes and gradient
    c = qi.grid_circuit(3, 3, 12, 4, param=True)
    bits = qi.bitstrings(c.n, 16, 4)
    plan = q.Plan(q.Model(q.Circuit.grid(3, 3, 12, 4, True)), batch=16, gradients=True).bind()
    d_bits = torch.from_numpy(bits.astype(np.int64)).cuda()
    th, ph = OG.params(c)
    for shift in (0.0, 0.3):
        c2 = c.with_angles(th + shift, ph - shift)
        params = torch.tensor(np.stack([th + shift, ph - shift], axis=1).reshape(-1), dtype=torch.float64,
                              requires_grad=True)
        a = q.autograd.amplitudes(plan, params, d_bits)
        assert np.max(np.abs(a.detach().cpu().numpy() - sv.amplitudes(c2, bits))) * 2 ** (c.n / 2) < 1e-5
        torch.sum(torch.log(torch.abs(a) ** 2)).backward()
        ok, worst = close(params.grad.numpy(), OG.grad_exact(c2, bits))
        assert ok, (shift, worst)


def test_sliced_gradient_equals_unsliced(q):
    # a sliced gradient plan recomputes each slice's forward intermediates
    # before its adjoint pass and adds the slices' shares
    c = qi.grid_circuit(4, 5, 20, 2, param=True)
    bits = qi.bitstrings(c.n, 8, 2)
    m = q.Model(q.Circuit.grid(4, 5, 20, 2, True))
    full = q.Plan(m, batch=8, gradients=True, executor=1)
    sliced = q.Plan(m, batch=8, gradients=True, executor=1, mem_budget_bytes=full.info.arena_bytes // 3)
    assert full.info.n_slices == 1 and 2 <= sliced.info.n_slices <= 64
    a_ref = sv.amplitudes(c, bits)
    w = a_ref / np.abs(a_ref) ** 2
    ww = np.zeros(16)
    ww[0::2], ww[1::2] = w.real, w.imag
    d_w = torch.from_numpy(ww).cuda()
    d_bits = torch.from_numpy(bits.astype(np.int64)).cuda()
    out = []
    for plan in (full, sliced):
        plan.bind()
        d_grad = torch.zeros(2 * len(c.param_gates), dtype=torch.float64, device="cuda")
        d_amp = torch.zeros(16, dtype=torch.float64, device="cuda")
        plan.amplitude_grad(d_bits, d_w, d_grad, d_amp)
        torch.cuda.synchronize()
        assert plan.status() == 0
        o = d_amp.cpu().numpy()
        assert np.max(np.abs(o[0::2] + 1j * o[1::2] - a_ref)) * 2 ** (c.n / 2) < 1e-5
        out.append(d_grad.cpu().numpy())
    ok, worst = close(out[1], out[0])
    assert ok, worst
    ok, worst = close(out[1], OG.grad_exact(c, bits))
    assert ok, worst


def test_gradient_needs_gradient_plan(q):
    plan = q.Plan(q.Model(q.Circuit.grid(3, 3, 8, 0, True)), batch=4).bind()
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    bits = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(q.QgmError):
        plan.amplitude_grad(bits, d, d)

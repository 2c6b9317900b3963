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


def test_grid6x6_d20_b256_param_sampled(q):
    # 6x6 grid, depth 20, parametrised angles, 256 bitstrings: the loss is
    # sum log|a|^2 over two of them (weights zero elsewhere); 8 sampled
    # parameters against the oracle's derivative insertion
    c = qi.grid_circuit(6, 6, 20, 0, param=True)
    bits = qi.bitstrings(c.n, 256, 0)
    sel = [3, 200]
    a_ref = ve.amplitudes(c, bits[sel])
    weights = np.zeros(256, dtype=complex)
    weights[sel] = a_ref / np.abs(a_ref) ** 2
    g, a = gpu_grad(q, c, bits, weights)
    assert np.max(np.abs(a[sel] - a_ref)) * 2 ** (c.n / 2) < 1e-5
    rng = np.random.default_rng(0)
    picks = rng.choice(len(g), 8, replace=False)
    ref_all = np.zeros(len(g))
    for qi_ in picks:
        p, w = divmod(int(qi_), 2)
        da = np.array([OG.amplitude_derivative_ve(c, int(bits[s]), p, w) for s in sel])
        ref_all[qi_] = 2 * np.real(np.sum(np.conj(weights[sel]) * da))
    ok, worst = close(g[picks], ref_all[picks])
    assert ok, worst


def test_gradient_needs_gradient_plan(q):
    plan = q.Plan(q.Model(q.Circuit.grid(3, 3, 8, 0, True)), batch=4).bind()
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    bits = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(q.QgmError):
        plan.amplitude_grad(bits, d, d)

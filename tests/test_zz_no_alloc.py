"""The allocation-free entry point, qgm_amplitudes_static, through the C ABI.

It serves callers that cannot allocate device memory when they need
amplitudes (a framework whose pool allocator owns the device memory, or a
latency-critical loop where cudaMalloc/cudaFree would synchronise the device):
its scratch is one static device array instead of a bound workspace.  It must
give the amplitudes of the ordinary entry point, qgm_amplitudes, on
consecutive calls (the array keeps the previous call's contents).  This file
is collected last so a failure here stops a -x run after every other test.
"""
import numpy as np
import pytest

import qgm_inputs as qi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-5   # the parity tests' tolerance
ABS_TOL = 1e-5   # on |a - a_ref| * 2^{n/2}


@pytest.fixture(scope="module")
def q():
    from paper_1712_05384_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1712_05384_gb300 as q
    q.lib()
    return q


def _as_complex(t):
    o = t.cpu().numpy()
    return o[0::2] + 1j * o[1::2]


def _close(a, ref, n):
    big = np.abs(ref) >= 2.0 ** (-n / 2)
    rel = np.max(np.abs(a - ref)[big] / np.abs(ref[big])) if big.any() else 0.0
    return rel < REL_TOL and np.max(np.abs(a - ref)) * 2.0 ** (n / 2) < ABS_TOL


def _bound(q, plan, d_bits, B, n_out):
    """Amplitudes from the ordinary entry point with a bound workspace."""
    plan.bind()
    out = torch.zeros(2 * n_out, dtype=torch.float64, device="cuda")
    plan.amplitudes(d_bits, out, B=B)
    torch.cuda.synchronize()
    assert plan.status() == 0
    return _as_complex(out)


def _static(q, plan, d_bits, B, n_out):
    out = torch.full((2 * n_out,), float("nan"), dtype=torch.float64, device="cuda")
    q._lib.check(q.lib().qgm_amplitudes_static(plan._h, d_bits.data_ptr(), B, out.data_ptr(), None))
    torch.cuda.synchronize()
    return _as_complex(out)


def test_static_scratch_matches_bound_workspace(q):
    # three plans that exercise what the static path does differently: a
    # plain one (4x4 depth 12), one with a GEMM-shaped step (4x5 depth 30,
    # run here on the FP32 cores; the bound reference is told to do the same)
    # and one sliced into 8 parts (the per-slice loop); called twice in a
    # row, with another plan's call in between leaving its tables behind
    cases = []
    for rows, cols, depth, B, kw in [(4, 4, 12, 50, {}), (4, 5, 30, 4, {"precision": "fp32", "order_kind": 1}),
                                     (4, 5, 30, 4, {"precision": "fp32", "order_kind": 1, "div": 4})]:
        kw = dict(kw)
        div = kw.pop("div", 0)
        m = q.Model(q.Circuit.grid(rows, cols, depth, 3))
        if div:
            full = q.Plan(m, batch=B, executor=q.EXEC_STEPWISE, **kw)
            kw["mem_budget_bytes"] = full.info.arena_bytes // div
        plan = q.Plan(m, batch=B, executor=q.EXEC_STEPWISE, **kw)
        assert plan.info.workspace_bytes <= (64 << 20)
        bits = qi.bitstrings(rows * cols, B, 3)
        d_bits = torch.from_numpy(bits.astype(np.int64)).cuda()
        cases.append((plan, d_bits, B, rows * cols))
    assert cases[1][0].info.n_gemm_steps > 0 and cases[2][0].info.n_slices > 1
    other = q.Plan(q.Model(q.Circuit.grid(3, 3, 9, 1)), batch=8)
    o_bits = torch.from_numpy(qi.bitstrings(9, 8, 1).astype(np.int64)).cuda()
    o_ref = _bound(q, other, o_bits, 8, 8)
    for plan, d_bits, B, n in cases:
        ref = _bound(q, plan, d_bits, B, B)
        for call in range(2):
            a = _static(q, plan, d_bits, B, B)
            assert _close(a, ref, n), f"{n} qubits, call {call}"
            o = _static(q, other, o_bits, 8, 8)
            assert _close(o, o_ref, 9), f"interleaved plan, call {call}"


def test_static_scratch_rejects_large_plans(q):
    # 6x6 depth 25 with 1000 bitstrings needs gigabytes of scratch
    big = q.Plan(q.Model(q.Circuit.grid(6, 6, 25, 0)), batch=1000)
    assert big.info.workspace_bytes > (64 << 20)
    d_bits = torch.zeros(1000, dtype=torch.int64, device="cuda")
    out = torch.zeros(2000, dtype=torch.float64, device="cuda")
    rc = q.lib().qgm_amplitudes_static(big._h, d_bits.data_ptr(), 1000, out.data_ptr(), None)
    assert rc == -2  # QGM_ERR_OOM
    assert b"static scratch" in q.lib().qgm_last_error()

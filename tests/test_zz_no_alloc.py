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


def test_static_scratch_matches_bound_workspace(q):
    B = 50
    bits = qi.bitstrings(16, B, 3)
    d_bits = torch.from_numpy(bits.astype(np.int64)).cuda()
    plan = q.Plan(q.Model(q.Circuit.grid(4, 4, 12, 3)), batch=B, executor=q.EXEC_STEPWISE)
    assert plan.info.workspace_bytes <= (64 << 20)
    # the ordinary entry point, with a caller-allocated workspace
    plan.bind()
    ref_out = torch.zeros(2 * B, dtype=torch.float64, device="cuda")
    plan.amplitudes(d_bits, ref_out)
    torch.cuda.synchronize()
    ref = _as_complex(ref_out)
    # a second plan on the static scratch in between leaves its tables behind
    other = q.Plan(q.Model(q.Circuit.grid(3, 3, 9, 1)), batch=8)
    o_bits = torch.from_numpy(qi.bitstrings(9, 8, 1).astype(np.int64)).cuda()
    o_out = torch.zeros(16, dtype=torch.float64, device="cuda")
    for call in range(2):
        out = torch.full((2 * B,), float("nan"), dtype=torch.float64, device="cuda")
        q._lib.check(q.lib().qgm_amplitudes_static(plan._h, d_bits.data_ptr(), B, out.data_ptr(),
                                                   None))
        torch.cuda.synchronize()
        a = _as_complex(out)
        assert _close(a, ref, 16), f"call {call}"
        q._lib.check(q.lib().qgm_amplitudes_static(other._h, o_bits.data_ptr(), 8,
                                                   o_out.data_ptr(), None))
        torch.cuda.synchronize()


def test_static_scratch_rejects_large_plans(q):
    # 6x6 depth 25 with 1000 bitstrings needs gigabytes of scratch
    big = q.Plan(q.Model(q.Circuit.grid(6, 6, 25, 0)), batch=1000)
    assert big.info.workspace_bytes > (64 << 20)
    d_bits = torch.zeros(1000, dtype=torch.int64, device="cuda")
    out = torch.zeros(2000, dtype=torch.float64, device="cuda")
    rc = q.lib().qgm_amplitudes_static(big._h, d_bits.data_ptr(), 1000, out.data_ptr(), None)
    assert rc == -2  # QGM_ERR_OOM
    assert b"static scratch" in q.lib().qgm_last_error()

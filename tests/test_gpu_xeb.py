"""Cross-entropy benchmarking and sampling from a computed set on the GPU
(App. B, C) against the oracle, on amplitudes of the 5x5 depth-20 circuit."""
import numpy as np
import pytest

import qgm_inputs as qi
from oracle import xeb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amps():
    from paper_1712_05384_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1712_05384_gb300 as q
    bits = qi.bitstrings(25, 1024, 0)
    p = q.Plan(q.Model(q.Circuit.grid(5, 5, 20, 0)), batch=1024).bind()
    d_bits = torch.from_numpy(bits.astype(np.int64)).cuda()
    d_out = torch.empty(2048, dtype=torch.float64, device="cuda")
    p.amplitudes(d_bits, d_out)
    torch.cuda.synchronize()
    return q, d_out


def test_xeb_stats_match_oracle(amps):
    q, d_out = amps
    scratch = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = q._lib.xeb_stats(d_out, 1024, 25, scratch)
    o = d_out.cpu().numpy()
    ref = xeb.stats(o[0::2] + 1j * o[1::2], 25)
    for k in ref:
        assert abs(st[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), k
    # uniform bitstrings are uncorrelated with p_U: alpha ~ 0 (statistical)
    assert abs(st["alpha"]) < 0.2


def test_sampling_matches_oracle_and_gives_ideal_cross_entropy(amps):
    q, d_out = amps
    m = 20000
    scratch = torch.zeros(1024, dtype=torch.float64, device="cuda")
    d_idx = torch.zeros(m, dtype=torch.int64, device="cuda")
    q._lib.sample_from_set(d_out, 1024, m, 7, scratch, d_idx)
    torch.cuda.synchronize()
    idx = d_idx.cpu().numpy()
    o = d_out.cpu().numpy()
    a = o[0::2] + 1j * o[1::2]
    ref, u, cdf = xeb.sample_from_set(a, m, 7)
    assert np.array_equal(idx, ref)
    # App. C: samples from the computed set reproduce the ideal cross entropy
    # (alpha ~ 1 up to O(1/sqrt(t)) with t = 1024 computed probabilities)
    st = xeb.stats(a[idx], 25)
    assert abs(st["alpha"] - 1) < 0.25

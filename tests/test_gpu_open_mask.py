"""Partially open outputs (Eq. psi_x with the deltas of k chosen outputs
omitted) through the C ABI, against the FP64 oracle (needs a GB300).

Entry b * 2^k + c of a batch is the amplitude of bitstring x_b with its open
qubits replaced by the bits of c (bit i of c = the i-th lowest open qubit).
Tolerances as in the batch parity tests.
"""
import os

import numpy as np
import pytest

import errmeasure
import qgm_inputs as qi
from oracle import statevector as sv
from oracle import ve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-5
ABS_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1712_05384_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def Q():
    import paper_1712_05384_gb300 as q
    return q


def errors(a, ref, n):
    return errmeasure.errors(a, ref, n, os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0])


def expand(bits, open_qubits):
    """Bitstrings x_b with their open qubits set from c, in output order."""
    k = len(open_qubits)
    out = np.empty((len(bits), 1 << k), dtype=np.uint64)
    clear = np.uint64(~sum(1 << q for q in open_qubits) & ((1 << 64) - 1))
    for c in range(1 << k):
        set_bits = sum(((c >> i) & 1) << q for i, q in enumerate(sorted(open_qubits)))
        out[:, c] = (bits & clear) | np.uint64(set_bits)
    return out


def device_amplitudes(p, bits):
    d_bits = torch.from_numpy(bits.astype(np.int64)).cuda()
    d_out = torch.empty(2 * (len(bits) << p.n_open), dtype=torch.float64, device="cuda")
    p.amplitudes(d_bits, d_out, B=len(bits))
    torch.cuda.synchronize()
    assert p.status() == 0
    o = d_out.cpu().numpy()
    return (o[0::2] + 1j * o[1::2]).reshape(len(bits), 1 << p.n_open)


@pytest.mark.parametrize("open_qubits", [[0], [1, 6, 13], [0, 3, 5, 10, 12, 15]])
def test_open_mask_4x4_d12_vs_state_vector(open_qubits):
    c = qi.grid_circuit(4, 4, 12, 0)
    q = Q()
    mask = sum(1 << j for j in open_qubits)
    p = q.Plan(q.Model(q.Circuit.grid(4, 4, 12, 0)), batch=16, open_mask=mask).bind()
    assert p.executor()[0] == 1          # resident executor keeps no open axes
    bits = qi.bitstrings(c.n, 13, 0)     # a ragged batch (13 of 16)
    a = device_amplitudes(p, bits)
    psi = sv.state(c)
    ref = psi[expand(bits, open_qubits).astype(np.int64)]
    rel, ab = errors(a.ravel(), ref.ravel(), c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)
    # the host entry point returns the same numbers, shaped (B, 2^k)
    h = p.amplitudes_host(bits)
    assert h.shape == (13, 1 << len(open_qubits))
    assert np.array_equal(h, a)


def test_open_mask_all_qubits_gives_the_state():
    # every output open: the final tensor has no batch axis and each row of
    # the output is the whole state, whatever the bitstring
    c = qi.grid_circuit(3, 3, 8, 2)
    q = Q()
    p = q.Plan(q.Model(q.Circuit.grid(3, 3, 8, 2)), batch=4, open_mask=(1 << 9) - 1).bind()
    bits = qi.bitstrings(c.n, 3, 2)
    a = device_amplitudes(p, bits)
    psi = sv.state(c)
    for row in a:
        rel, ab = errors(row, psi, c.n)
        assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)


def test_open_mask_5x5_d20_sampled_and_consistent_with_closed_plan():
    # 64 bitstrings x 2^4 open outputs of the 5x5 depth-20 workload: sampled
    # entries against the oracle's elimination, every entry against the
    # closed batch plan run on the expanded bitstrings
    c = qi.grid_circuit(5, 5, 20, 0)
    q = Q()
    open_qubits = [2, 7, 12, 24]
    m = q.Model(q.Circuit.grid(5, 5, 20, 0))
    p = q.Plan(m, batch=64, open_mask=sum(1 << j for j in open_qubits)).bind()
    bits = qi.bitstrings(c.n, 64, 0)
    a = device_amplitudes(p, bits)
    full = expand(bits, open_qubits).ravel()
    closed = q.Plan(m, batch=len(full), executor=1).bind()
    b = device_amplitudes(closed, full).ravel()
    rel, ab = errors(a.ravel(), b, c.n)
    assert rel < 2 * REL_TOL and ab < 2 * ABS_TOL, (rel, ab)
    idx = np.linspace(0, len(full) - 1, 24).astype(int)
    ref = ve.amplitudes(c, full[idx])
    rel, ab = errors(a.ravel()[idx], ref, c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)


def test_open_mask_with_slicing():
    # a memory budget that forces slicing: the slices sum into the same
    # B x 2^k outputs
    c = qi.grid_circuit(4, 4, 12, 1)
    q = Q()
    m = q.Model(q.Circuit.grid(4, 4, 12, 1))
    mask = (1 << 4) | (1 << 11)
    full = q.Plan(m, batch=8, open_mask=mask)
    p = q.Plan(m, batch=8, open_mask=mask, mem_budget_bytes=full.info.arena_bytes // 2).bind()
    assert p.info.n_slices > 1
    bits = qi.bitstrings(c.n, 8, 1)
    a = device_amplitudes(p, bits)
    ref = sv.state(c)[expand(bits, [4, 11]).astype(np.int64)]
    rel, ab = errors(a.ravel(), ref.ravel(), c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)

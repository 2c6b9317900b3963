"""GEMM-shaped steps on the tensor cores (split 16-bit terms, tcgen05) against
the FP64 oracle and against the FP32-core GEMM kernel (needs a GB300).

Both split forms carry near-FP32 error: split FP16 writes each scaled FP32
value as h + l (22 significant bits) and keeps h h' + h l' + l h'; split
BF16 writes it as three 8-bit terms and keeps the six term products above
2^-24 of the product.  The bound asserted is the one stated for the split
form, 1e-4, on both error measures (relative over amplitudes with
|a_ref| >= 2^{-n/2}, and |a - a_ref| * 2^{n/2} over all of them); the
measured errors are printed (run with -s).
"""
import os

import numpy as np
import pytest

import errmeasure
import qgm_inputs as qi
from oracle import statevector as sv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPLIT_TOL = 1e-4
PRECISIONS = ["fp16", "bf16"]


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


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("rows,cols,depth,B,n_tc", [(4, 5, 30, 16, 1), (4, 6, 34, 6, 4)])
def test_split_gemm_vs_state_vector(rows, cols, depth, B, n_tc, precision):
    # 4x5 d30: one GEMM step, both operands batched (one product per batch
    # entry), 128 x 64 tiles; 4x6 d34: four of five GEMM steps on the tensor
    # cores -- two with one batch-free operand (the batch entries become rows
    # of the other; one with the roles exchanged), two with 4 summed entries
    # (zero-padded to one chunk of 16), one without a batch axis -- and the
    # fifth (2^6 rows on both sides, both batched) left to the FP32 kernel
    q = Q()
    c = qi.grid_circuit(rows, cols, depth, 0)
    bits = qi.bitstrings(c.n, B, 0)
    ref = sv.amplitudes(c, bits)
    p = q.Plan(q.Model(q.Circuit.grid(rows, cols, depth, 0)), order_kind=1, batch=B, executor=1,
               precision=precision)
    assert p.info.n_gemm_tc_steps == n_tc
    a = p.bind().amplitudes_host(bits)
    assert p.status() == 0
    rel, ab = errors(a, ref, c.n)
    assert rel < SPLIT_TOL and ab < SPLIT_TOL, (rel, ab)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_split_matches_fp32_gemm_4x8_d40(precision):
    # 4x8 depth 40, 4 bitstrings: four GEMM steps (one folded with roles
    # exchanged, one folded, two per entry, one of those with 4 summed
    # entries); no oracle runs 32 qubits at depth 40 in a test, so the
    # FP32-core GEMM plan is the comparison (it is checked against the oracle
    # at smaller sizes)
    q = Q()
    m = q.Model(q.Circuit.grid(4, 8, 40, 0))
    bits = qi.bitstrings(32, 4, 0)
    pt = q.Plan(m, order_kind=1, batch=4, precision=precision)
    assert pt.info.n_gemm_tc_steps == pt.info.n_gemm_steps == 4
    a = pt.bind().amplitudes_host(bits)
    assert pt.status() == 0
    b = q.Plan(m, order_kind=1, batch=4, precision="fp32").bind().amplitudes_host(bits)
    rel, ab = errors(a, b, 32)
    assert rel < SPLIT_TOL and ab < SPLIT_TOL, (rel, ab)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_split_narrow_tiles_with_wide_batch(precision):
    # 4x6 depth 30, 64 bitstrings, contraction trees: GEMM steps with narrow
    # N tiles and a 64-entry batch axis; against the product-sum kernels (no
    # GEMM) and the oracle
    q = Q()
    c = qi.grid_circuit(4, 6, 30, 0)
    bits = qi.bitstrings(c.n, 64, 0)
    m = q.Model(q.Circuit.grid(4, 6, 30, 0))
    p = q.Plan(m, batch=64, trees=True, executor=1, precision=precision)
    assert p.info.n_gemm_tc_steps == p.info.n_gemm_steps >= 1
    a = p.bind().amplitudes_host(bits)
    assert p.status() == 0
    b = q.Plan(m, batch=64, trees=True, executor=1, gemm=False).bind().amplitudes_host(bits)
    rel, ab = errors(a, b, c.n)
    assert rel < SPLIT_TOL and ab < SPLIT_TOL, (rel, ab)
    from oracle import ve
    rel, ab = errors(a[:4], ve.amplitudes(c, bits[:4]), c.n)
    assert rel < SPLIT_TOL and ab < SPLIT_TOL, (rel, ab)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_in_kernel_conversion_matches_split_pass(precision):
    # folded steps (batch entries as rows of M): converting the batched
    # operand inside the product kernel gives the same terms as the split
    # pass, so the same bits; 4x6 d34 against the oracle, 4x8 d40 pairwise
    q = Q()
    c = qi.grid_circuit(4, 6, 34, 0)
    bits = qi.bitstrings(c.n, 6, 0)
    m = q.Model(q.Circuit.grid(4, 6, 34, 0))
    a = q.Plan(m, order_kind=1, batch=6, executor=1, precision=precision, tc_convert=True)
    assert any(g["conv_ok"] for g in a.gemm_shapes())
    a = a.bind()
    b = q.Plan(m, order_kind=1, batch=6, executor=1, precision=precision).bind()
    assert np.array_equal(a.amplitudes_host(bits), b.amplitudes_host(bits))
    rel, ab = errors(a.amplitudes_host(bits), sv.amplitudes(c, bits), c.n)
    assert rel < SPLIT_TOL and ab < SPLIT_TOL, (rel, ab)
    m = q.Model(q.Circuit.grid(4, 8, 40, 0))
    bits = qi.bitstrings(32, 4, 0)
    pa = q.Plan(m, order_kind=1, batch=4, precision=precision, tc_convert=True)
    assert any(g["conv_ok"] for g in pa.gemm_shapes())
    a = pa.bind().amplitudes_host(bits)
    b = q.Plan(m, order_kind=1, batch=4, precision=precision).bind().amplitudes_host(bits)
    assert np.array_equal(a, b)


def test_repeat_calls_are_identical():
    # the planes are rewritten on every call: two calls give the same bits
    q = Q()
    m = q.Model(q.Circuit.grid(4, 6, 34, 0))
    bits = qi.bitstrings(24, 6, 0)
    p = q.Plan(m, order_kind=1, batch=6, executor=1).bind()
    a = p.amplitudes_host(bits)
    b = p.amplitudes_host(bits[::-1].copy())
    c = p.amplitudes_host(bits)
    assert np.array_equal(a, c)
    assert np.max(np.abs(a - b[::-1])) <= 1e-12 * np.max(np.abs(a))


@pytest.mark.parametrize("rows,cols,depth,B,trees", [(4, 6, 34, 6, None), (4, 6, 30, 64, True)])
def test_every_tuning_candidate_gives_the_same_amplitudes(rows, cols, depth, B, trees):
    # the autotuner's candidates (tensor-core N tile, in-kernel conversion,
    # product-sum term groups and terms in flight) compute the same products:
    # each setting, applied to every step by hand, matches the fixed rules
    # and the oracle
    q = Q()
    c = qi.grid_circuit(rows, cols, depth, 0)
    bits = qi.bitstrings(c.n, B, 0)
    m = q.Model(q.Circuit.grid(rows, cols, depth, 0))
    p = q.Plan(m, order_kind=1, batch=B, executor=1, trees=trees).bind()
    base = p.amplitudes_host(bits)
    from oracle import ve
    ref = ve.amplitudes(c, bits[:4])
    n_steps = p.info.n_steps
    with pytest.raises(q.QgmError):
        p.set_tuning([{"step": 0, "nt_cap": 100}])
    for nt in (64, 128, 256):
        for conv in (0, 1):
            for T in (1, 2, 4):
                for U in (2, 4, 8):
                    p.set_tuning([{"step": s, "nt_cap": nt, "conv": conv, "T": T, "U": U} for s in range(n_steps)])
                    a = p.amplitudes_host(bits)
                    assert p.status() == 0
                    scale = np.max(np.abs(base))
                    assert np.max(np.abs(a - base)) <= 1e-5 * scale, (nt, conv, T, U)
                    rel, ab = errmeasure.measures(a[:4], ref, c.n)["rel"], errmeasure.measures(a[:4], ref, c.n)["abs"]
                    assert rel < SPLIT_TOL and ab < SPLIT_TOL, (nt, conv, T, U, rel, ab)
    got = p.tuning()
    assert len(got) == n_steps and all(t["U"] == 8 and t["T"] == 4 for t in got)
    # GEMM-shaped steps as product-sums (where no tensor keeps its batch
    # entry outermost; the others refuse)
    shapes = p.gemm_shapes()
    ok = [g["step"] for g in shapes if not g["o_bout"] and not g["in_bout"]]
    assert ok
    for U in (2, 4):
        p.set_tuning([{"step": s, "ps": 1, "U": U} for s in ok])
        a = p.amplitudes_host(bits)
        assert p.status() == 0
        assert np.max(np.abs(a - base)) <= 1e-5 * np.max(np.abs(base)), U
    bout = [g["step"] for g in shapes if g["o_bout"] or g["in_bout"]]
    if bout:
        with pytest.raises(q.QgmError):
            p.set_tuning([{"step": bout[0], "ps": 1}])

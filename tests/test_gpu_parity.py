"""CUDA path vs the FP64 oracle, through the C ABI (needs a GB300).

Tolerance (complex64 path): the paper reports relative error below 1e-5 per
probability in single precision.  FP32 elimination has an absolute error
floor proportional to the root-mean-square amplitude 2^{-n/2}, so relative
error is taken over amplitudes with |a_ref| >= 2^{-n/2} (probability at least
the uniform 2^{-n}; about 37% of outputs under Porter-Thomas) and, over ALL
amplitudes, the error relative to the rms amplitude, |a - a_ref| * 2^{n/2}.
Both must stay below 1e-5.
"""
import json
import math
import os

import numpy as np
import pytest

import errmeasure
import qgm_inputs as qi
from oracle import statevector as sv
from oracle import ve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EXECS = [1, 2, 3]   # stepwise, resident, compiled resident
REL_TOL = 1e-5
ABS_TOL = 1e-5   # on |a - a_ref| * 2^{n/2}


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


def run_batch(circuit_py, B, order_kind=0, budget=0, bits=None, max_fuse=0, executor=0, trees=False):
    q = Q()
    if circuit_py.rows:
        c = q.Circuit.grid(circuit_py.rows, circuit_py.cols, circuit_py.depth, circuit_py.seed,
                           circuit_py.param)
    else:
        c = q.Circuit.from_gates(circuit_py.n, circuit_py.gates)
    p = q.Plan(q.Model(c), order_kind=order_kind, batch=B, mem_budget_bytes=budget,
               max_fuse=max_fuse, executor=executor, trees=trees).bind()
    if executor:
        assert p.executor()[0] == executor
    if bits is None:
        bits = qi.bitstrings(circuit_py.n, B, circuit_py.seed)
    d_bits = torch.from_numpy(bits.astype(np.int64)).cuda()
    d_out = torch.empty(2 * len(bits), dtype=torch.float64, device="cuda")
    p.amplitudes(d_bits, d_out, B=len(bits))
    torch.cuda.synchronize()
    assert p.status() == 0
    o = d_out.cpu().numpy()
    return o[0::2] + 1j * o[1::2], bits, p


@pytest.mark.parametrize("executor", EXECS)
def test_app_d_example(app_d, executor):
    a, bits, _ = run_batch(app_d, 4, bits=np.arange(4, dtype=np.uint64), executor=executor)
    ref = sv.state(app_d)
    assert abs(a[0] - 0.5) < 1e-7          # App. D: <00|C|00> = 1/2
    assert np.allclose(a, ref, atol=1e-7)


@pytest.mark.parametrize("executor", EXECS)
@pytest.mark.parametrize("rows,cols,depth,B", [(3, 3, 8, 37), (4, 4, 12, 64), (2, 5, 16, 5),
                                               (3, 4, 20, 130)])
def test_small_grids_vs_state_vector(rows, cols, depth, B, executor):
    c = qi.grid_circuit(rows, cols, depth, seed=2)
    a, bits, _ = run_batch(c, B, executor=executor)
    ref = sv.amplitudes(c, bits)
    rel, ab = errors(a, ref, c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)


@pytest.mark.parametrize("executor", EXECS)
@pytest.mark.parametrize("kind", [1, 2, 3])
def test_every_order_kind(kind, executor):
    c = qi.grid_circuit(4, 4, 14, seed=5)
    a, bits, p = run_batch(c, 48, order_kind=kind, executor=executor)
    assert p.info.order_kind == kind
    rel, ab = errors(a, sv.amplitudes(c, bits), c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)


def test_sliced_equals_unsliced():
    c = qi.grid_circuit(4, 5, 16, seed=1)
    a0, bits, p0 = run_batch(c, 40, order_kind=1)
    a1, _, p1 = run_batch(c, 40, order_kind=1, budget=p0.info.arena_bytes // 5)
    assert p1.info.n_slices > 1
    rel, ab = errors(a1, sv.amplitudes(c, bits), c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)
    assert np.max(np.abs(a1 - a0)) * 2 ** (c.n / 2) < 1e-5


@pytest.mark.parametrize("executor", EXECS)
def test_fusion_limits_agree(executor):
    c = qi.grid_circuit(4, 4, 16, seed=9)
    a1, bits, _ = run_batch(c, 24, max_fuse=1, executor=executor)
    a8, _, _ = run_batch(c, 24, max_fuse=8, executor=executor)
    ref = sv.amplitudes(c, bits)
    for a in (a1, a8):
        rel, ab = errors(a, ref, c.n)
        assert rel < REL_TOL and ab < ABS_TOL


@pytest.mark.parametrize("executor", EXECS)
def test_parametrised_circuit(executor):
    c = qi.grid_circuit(3, 4, 14, seed=4, param=True)
    a, bits, _ = run_batch(c, 33, executor=executor)
    rel, ab = errors(a, sv.amplitudes(c, bits), c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)


@pytest.mark.parametrize("executor", EXECS)
def test_depth_one_is_uniform(executor):
    # only the H layer: every amplitude is 2^{-n/2}
    c = qi.grid_circuit(3, 3, 1, seed=0)
    a, _, _ = run_batch(c, 12, executor=executor)
    assert np.allclose(a, 2 ** -4.5, rtol=1e-7, atol=0)


def test_open_outputs_4x4_d10_all_amplitudes():
    # 4x4 grid, depth 10: all 2^16 amplitudes at once (output deltas omitted)
    q = Q()
    c = qi.grid_circuit(4, 4, 10, 0)
    p = q.Plan(q.Model(q.Circuit.grid(4, 4, 10, 0)), output_mode=q.OUT_OPEN).bind()
    d_out = torch.empty(2 << 16, dtype=torch.float64, device="cuda")
    p.eliminate(d_out)
    torch.cuda.synchronize()
    o = d_out.cpu().numpy()
    a = o[0::2] + 1j * o[1::2]
    ref = sv.state(c)
    rel, ab = errors(a, ref, c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)
    assert abs(np.vdot(a, a).real - 1) < 1e-5
    assert np.allclose(a, ve.open_amplitudes(c), atol=1e-6 * 2 ** -8)


@pytest.mark.parametrize("executor", [0, 1])
def test_grid5x5_d20_b1024_sampled(executor):
    # full-size workload; executor 0 (auto) is the launch configuration the
    # benchmark times; 64 sampled outputs against the oracle's own elimination
    c = qi.grid_circuit(5, 5, 20, 0)
    a, bits, p = run_batch(c, 1024, executor=executor)
    if executor == 0:
        assert p.executor()[0] == 3
    idx = np.linspace(0, 1023, 64).astype(int)
    ref = ve.amplitudes(c, bits[idx])
    rel, ab = errors(a[idx], ref, c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)
    # over uniform x, E[N p] = sum_x p_x = 1 exactly, and E[(N p)^2] is the
    # collision moment N sum p^2 of this circuit (2.458 from the oracle's
    # state vector; Porter-Thomas would give 2): 4-sigma sample bands
    Np = (2 ** c.n) * np.abs(a) ** 2
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "moments_grid5x5_d20.json")))
    assert abs(Np.mean() - 1) < 4 * Np.std() / math.sqrt(len(Np))
    assert abs((Np ** 2).mean() - gold["N_sum_p2"]) < 4 * (Np ** 2).std() / math.sqrt(len(Np))


def _golden(name):
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        return json.load(f)


@pytest.mark.parametrize("precision", ["fp16", "bf16", "fp32"])
def test_grid6x6_d25_b1000_vs_oracle(precision):
    # 6x6 grid, depth 25, the full batch of 1000 bitstrings (intermediates up
    # to 2^28 complex64 entries, stepwise executor); its first 32 outputs
    # against the FP64 oracle's values (tests/golden/amps_grid6x6_d25.json,
    # oracle/ve.c); the GEMM step on the tensor cores in split FP16 or BF16,
    # or every GEMM step on the FP32 cores
    gold = _golden("amps_grid6x6_d25.json")
    q = Q()
    c = qi.grid_circuit(6, 6, 25, 0)
    bits = qi.bitstrings(c.n, 1000, 0)
    p = q.Plan(q.Model(q.Circuit.grid(6, 6, 25, 0)), batch=1000, precision=precision).bind()
    assert p.info.max_tensor_entries >= 2 ** 26
    assert (p.info.n_gemm_tc_steps > 0) == (precision != "fp32")
    d_bits = torch.from_numpy(bits.astype(np.int64)).cuda()
    d_out = torch.empty(2000, dtype=torch.float64, device="cuda")
    p.amplitudes(d_bits, d_out)
    torch.cuda.synchronize()
    assert p.status() == 0
    o = d_out.cpu().numpy()
    a = o[0::2] + 1j * o[1::2]
    xs = [int(e["x"]) for e in gold["amplitudes"]]
    assert len(xs) >= 32 and xs == [int(x) for x in bits[:len(xs)]]
    ref = np.array([complex(e["re"], e["im"]) for e in gold["amplitudes"]])
    rel, ab = errors(a[:len(xs)], ref, c.n)
    tol = REL_TOL if precision == "fp32" else 1e-4
    assert rel < tol and ab < tol, (rel, ab)
    Np = (2 ** c.n) * np.abs(a) ** 2
    assert abs(Np.mean() - 1) < 4 * Np.std() / math.sqrt(len(Np))


@pytest.mark.parametrize("precision", ["fp16", "bf16", "fp32"])
def test_grid5x9_d40_vs_oracle(precision):
    # 5x9 grid, depth 40, in passes of 4 bitstrings (the benchmark's plan):
    # the first outputs of the seed-0 batch against the FP64 oracle's values
    # (tests/golden/amps_grid5x9_d40.json: oracle/ve.c, sliced, hours of CPU);
    # complex64 (GEMM steps on the FP32 cores) within 1e-5, the split forms
    # within 1e-4
    path = os.path.join(os.path.dirname(__file__), "golden", "amps_grid5x9_d40.json")
    if not os.path.exists(path):
        pytest.skip("no oracle amplitudes stored for 5x9 depth 40")
    gold = _golden("amps_grid5x9_d40.json")
    xs = [int(e["x"]) for e in gold["amplitudes"]]
    if len(xs) < 2:
        pytest.skip("fewer than two oracle amplitudes stored")
    q = Q()
    bits = qi.bitstrings(45, 1000, 0)
    assert xs == [int(x) for x in bits[:len(xs)]]
    p = q.Plan(q.Model(q.Circuit.grid(5, 9, 40, 0)), order_kind=1, batch=4, precision=precision).bind()
    assert p.info.n_gemm_steps > 0 and (p.info.n_gemm_tc_steps > 0) == (precision != "fp32")
    a = np.concatenate([p.amplitudes_host(bits[k:k + 4]) for k in range(0, len(xs), 4)])[:len(xs)]
    assert p.status() == 0
    ref = np.array([complex(e["re"], e["im"]) for e in gold["amplitudes"]])
    rel, ab = errors(a, ref, 45)
    tol = REL_TOL if precision == "fp32" else 1e-4
    assert rel < tol and ab < tol, (rel, ab)


@pytest.mark.parametrize("executor", EXECS)
def test_host_api_matches_device_api(executor):
    q = Q()
    c = qi.grid_circuit(4, 4, 12, 3)
    bits = qi.bitstrings(16, 50, 3)
    a_dev, _, p = run_batch(c, 50, bits=bits, executor=executor)
    a_host = p.amplitudes_host(bits)
    assert np.array_equal(a_dev, a_host)
    # a second call with fewer bitstrings reuses the plan
    a_part = p.amplitudes_host(bits[:7])
    assert np.array_equal(a_part, a_dev[:7])


def test_errors_are_reported():
    q = Q()
    m = q.Model(q.Circuit.grid(3, 3, 8, 0))
    p = q.Plan(m, batch=8)
    d_bits = torch.zeros(8, dtype=torch.int64, device="cuda")
    d_out = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QgmError):
        p.amplitudes(d_bits, d_out)               # not bound
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(q.QgmError):
        p.bind(small)                             # workspace too small
    p.bind()
    with pytest.raises(q.QgmError):
        p.amplitudes(d_bits, d_out, B=9)          # more than the plan's batch
    with pytest.raises(q.QgmError):
        p.eliminate(d_out)                        # not an open-output plan
    m2 = q.Model(q.Circuit.grid(4, 5, 16, 1))
    full = q.Plan(m2, order_kind=1, batch=8)
    sliced = q.Plan(m2, order_kind=1, batch=8, mem_budget_bytes=full.info.arena_bytes // 4)
    assert sliced.info.n_slices > 1
    with pytest.raises(q.QgmError):               # resident needs one slice
        q.Plan(m2, order_kind=1, batch=8, mem_budget_bytes=full.info.arena_bytes // 4,
               executor=2)


def test_bounded_wait_gives_timeout_status():
    # failure detection without a fault: the tensor-core kernels' bounded
    # mbarrier wait on a barrier nothing arrives at gives up after its limit
    # and reports QGM_ERR_TIMEOUT; the context stays usable afterwards
    import time
    q = Q()
    from paper_1712_05384_gb300 import _lib
    t0 = time.perf_counter()
    assert _lib.selftest_wait_timeout(200_000_000) == -4
    assert time.perf_counter() - t0 >= 0.2
    assert _lib.selftest_wait_timeout(200_000_000, arrive=True) == 0
    with pytest.raises(q.QgmError):
        _lib.selftest_wait_timeout(10)                 # limit out of range
    c = qi.grid_circuit(3, 3, 8, 0)
    bits = qi.bitstrings(c.n, 8, 0)
    a = q.Plan(q.Model(q.Circuit.grid(3, 3, 8, 0)), batch=8, executor=1).bind().amplitudes_host(bits)
    rel, ab = errors(a, sv.amplitudes(c, bits), c.n)
    assert rel < REL_TOL and ab < ABS_TOL


@pytest.mark.parametrize("executor", [2, 3])
@pytest.mark.parametrize("chunk", [1, 2, 4, 8])
def test_resident_chunks_agree(chunk, executor):
    # bitstrings per CTA 1..8, batch 77 leaves a ragged last chunk
    q = Q()
    c = qi.grid_circuit(4, 4, 16, 6)
    bits = qi.bitstrings(16, 77, 6)
    ref = sv.amplitudes(c, bits)
    p = q.Plan(q.Model(q.Circuit.grid(4, 4, 16, 6)), batch=77, executor=executor,
               resident_chunk=chunk).bind()
    assert p.executor()[:2] == (executor, chunk)
    a = p.amplitudes_host(bits)
    rel, ab = errors(a, ref, c.n)
    assert rel < REL_TOL and ab < ABS_TOL


@pytest.mark.parametrize("rows,cols,depth,B", [(4, 5, 30, 16), (4, 6, 34, 6)])
def test_gemm_steps_vs_state_vector(rows, cols, depth, B):
    # depths at which the plan has GEMM-shaped steps (two operands sharing
    # every summed variable); the tiled GEMM kernel and the product-sum
    # kernel must both agree with the state vector
    q = Q()
    c = qi.grid_circuit(rows, cols, depth, 0)
    bits = qi.bitstrings(c.n, B, 0)
    ref = sv.amplitudes(c, bits)
    # GEMM steps on the tensor cores (split BF16, the default), on the FP32
    # cores, and no GEMM steps (product-sum kernels)
    for gemm, split in ((True, None), (True, False), (False, None)):
        p = q.Plan(q.Model(q.Circuit.grid(rows, cols, depth, 0)), order_kind=1, batch=B,
                   executor=1, gemm=gemm, split_bf16=split)
        assert (p.info.n_gemm_steps > 0) == gemm
        assert (p.info.n_gemm_tc_steps > 0) == (gemm and split is None)
        a = p.bind().amplitudes_host(bits)
        rel, ab = errors(a, ref, c.n)
        assert rel < REL_TOL and ab < ABS_TOL, (gemm, split, rel, ab)


def test_grid5x9_d40_two_plans_and_porter_thomas():
    # 5x9 grid, depth 40: no oracle finishes it, so (1) the same amplitudes
    # from an unsliced and a sliced plan, (2) depth 16 of the same grid
    # against the oracle, (3) Porter-Thomas moments over 256 amplitudes
    q = Q()
    m = q.Model(q.Circuit.grid(5, 9, 40, 0))
    bits = qi.bitstrings(45, 256, 0)
    p1 = q.Plan(m, order_kind=1, batch=4)
    assert p1.info.n_gemm_steps > 0
    p1.bind()
    a1 = p1.amplitudes_host(bits[:4])
    p2 = q.Plan(m, order_kind=1, batch=4, mem_budget_bytes=p1.info.arena_bytes // 3)
    assert p2.info.n_slices > 1
    a2 = p2.bind().amplitudes_host(bits[:4])
    del p2
    assert np.max(np.abs(a1 - a2)) * 2 ** 22.5 < 1e-5
    c16 = qi.grid_circuit(5, 9, 16, 0)
    a16 = q.Plan(q.Model(q.Circuit.grid(5, 9, 16, 0)), batch=4).bind().amplitudes_host(bits[:4])
    rel, ab = errors(a16, ve.amplitudes(c16, bits[:4]), 45)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)
    A = np.concatenate([p1.amplitudes_host(bits[4 * k:4 * k + 4]) for k in range(64)])
    Np = 2 ** 45 * np.abs(A) ** 2
    se1, se2 = Np.std() / 16, (Np ** 2).std() / 16
    assert abs(Np.mean() - 1) < 4 * se1
    assert abs((Np ** 2).mean() - 2) < 4 * se2


@pytest.mark.parametrize("executor", EXECS)
def test_nonfinite_gate_sets_status(executor):
    # failure detection without a GPU fault: a NaN gate angle makes NaN
    # tables; the first tensor holding NaN is flagged through the status word
    q = Q()
    c = qi.grid_circuit(3, 3, 10, 1, param=True)
    gates = list(c.gates)
    g = gates[c.param_gates[0]]
    gates[c.param_gates[0]] = qi.Gate(g.kind, g.cycle, g.q0, g.q1, float("nan"), g.phi)
    p = q.Plan(q.Model(q.Circuit.from_gates(9, gates)), batch=8, executor=executor).bind()
    d_bits = torch.from_numpy(qi.bitstrings(9, 8, 1).astype(np.int64)).cuda()
    d_out = torch.empty(16, dtype=torch.float64, device="cuda")
    p.amplitudes(d_bits, d_out)
    torch.cuda.synchronize()
    assert p.status() == -5          # QGM_ERR_NONFINITE, and cleared by the read
    assert p.status() == 0


def test_register_tiled_steps_vs_state_vector():
    # 4x5 grid, depth 24, 1024 bitstrings on the stepwise executor: several
    # expanding steps run with a register tile; all amplitudes vs the state
    # vector, and identical to the plain batched kernel's up to rounding
    q = Q()
    c = qi.grid_circuit(4, 5, 24, 0)
    bits = qi.bitstrings(c.n, 1024, 0)
    p = q.Plan(q.Model(q.Circuit.grid(4, 5, 24, 0)), batch=1024, executor=1)
    assert p.info.n_tile_steps > 0
    a = p.bind().amplitudes_host(bits)
    rel, ab = errors(a, sv.amplitudes(c, bits), c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)


@pytest.mark.parametrize("executor", EXECS)
@pytest.mark.parametrize("rows,cols,depth,B", [(4, 4, 14, 40), (3, 5, 20, 17)])
def test_contraction_trees_vs_state_vector(rows, cols, depth, B, executor):
    # buckets run as contraction trees (pairs first, each variable summed as
    # soon as no other factor holds it): same amplitudes, fewer products
    c = qi.grid_circuit(rows, cols, depth, seed=7)
    a, bits, p = run_batch(c, B, executor=executor, trees=True)
    rel, ab = errors(a, sv.amplitudes(c, bits), c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)


def test_contraction_trees_grid5x5_d20_sampled():
    c = qi.grid_circuit(5, 5, 20, 0)
    a, bits, p = run_batch(c, 1024, trees=True)
    idx = np.linspace(0, 1023, 24).astype(int)
    rel, ab = errors(a[idx], ve.amplitudes(c, bits[idx]), c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)


def test_compiled_many_waves_runs_shared_part_once():
    # 4x4 depth 12 with 3000 bitstrings: several waves of one-bitstring CTAs,
    # so the compiled executor runs the steps without a batch axis once per
    # call in a kernel of their own, whose outputs every CTA reads
    c = qi.grid_circuit(4, 4, 12, 8)
    a, bits, p = run_batch(c, 3000, executor=3)
    assert p.executor()[:2] == (3, 1)
    rel, ab = errors(a, sv.amplitudes(c, bits), c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)


def test_compiled_grid6x6_d20_param_sampled():
    # the widest plan here that fits the resident executors (116 KB of shared
    # memory per bitstring): compiled kernel against the oracle on sampled
    # bitstrings, and against the stepwise executor on all 256
    c = qi.grid_circuit(6, 6, 20, 0, param=True)
    a3, bits, p3 = run_batch(c, 256, executor=3)
    assert p3.executor()[0] == 3
    a1, _, _ = run_batch(c, 256, executor=1)
    rel, ab = errors(a3, a1, c.n)
    assert rel < 2 * REL_TOL and ab < 2 * ABS_TOL, (rel, ab)
    idx = np.linspace(0, 255, 6).astype(int)
    rel, ab = errors(a3[idx], ve.amplitudes(c, bits[idx]), c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)


@pytest.mark.parametrize("executor", [2, 3])
def test_host_api_with_page_locked_buffers(executor):
    # page-locked host buffers are read and written in place by the resident
    # executors; pageable ones go through staging copies; same amplitudes
    import ctypes as C
    q = Q()
    c = qi.grid_circuit(4, 4, 12, 3)
    bits = qi.bitstrings(16, 50, 3)
    a_dev, _, p = run_batch(c, 50, bits=bits, executor=executor)
    hb = torch.from_numpy(bits.astype(np.int64)).pin_memory()
    ho = torch.zeros(100, dtype=torch.float64).pin_memory()
    for _ in range(2):
        ho.zero_()
        q._lib.check(q.lib().qgm_amplitudes_host(p._h, hb.data_ptr(), 50, ho.data_ptr(), None))
        o = ho.numpy()
        assert np.array_equal(o[0::2] + 1j * o[1::2], a_dev)
    assert np.array_equal(p.amplitudes_host(bits), a_dev)


def test_narrow_gemm_tiles_with_wide_batch():
    # 4x6 depth 30, 64 bitstrings, contraction trees, FP32-core GEMM: one
    # GEMM-shaped step has five private variables on one side and runs with
    # 64 x 32 tiles; the
    # amplitudes equal the product-sum kernels' (no GEMM) and the oracle's
    q = Q()
    c = qi.grid_circuit(4, 6, 30, 0)
    bits = qi.bitstrings(c.n, 64, 0)
    m = q.Model(q.Circuit.grid(4, 6, 30, 0))
    p = q.Plan(m, batch=64, trees=True, executor=1, split_bf16=False)
    assert p.info.n_gemm_steps > q.Plan(m, batch=8, trees=True, executor=1, precision="fp32").info.n_gemm_steps
    assert p.info.n_gemm_tc_steps == 0
    a = p.bind().amplitudes_host(bits)
    b = q.Plan(m, batch=64, trees=True, executor=1, gemm=False).bind().amplitudes_host(bits)
    rel, ab = errors(a, b, c.n)
    assert rel < 2 * REL_TOL and ab < 2 * ABS_TOL, (rel, ab)
    rel, ab = errors(a[:4], ve.amplitudes(c, bits[:4]), c.n)
    assert rel < REL_TOL and ab < ABS_TOL, (rel, ab)


def test_eliminate_fixed_app_d_tables(app_d):
    # App. D: with the inputs and outputs fixed to 0, eliminating b_1^1
    # leaves tau_2(b_0^1) = (1/2, 0) and summing b_0^1 gives <00|C|00> = 1/2.
    # qgm_eliminate_fixed returns the raw final tensor (times the plan's
    # constant) and its power-of-two exponent
    q = Q()
    c = q.Circuit.from_gates(app_d.n, app_d.gates)
    m = q.Model(c)
    qubit, k = m.vars()
    b01 = [v for v in range(len(qubit)) if qubit[v] == 0 and k[v] == 1][0]
    for executor in EXECS:
        p = q.Plan(m, batch=1, executor=executor)
        p.bind()
        raw, e = p.eliminate_fixed([0, 0])
        assert abs(raw[0] * 2.0 ** e - 0.5) < 1e-7
        pk = q.Plan(m, batch=1, keep_vars=[b01], executor=1).bind()
        raw, e = pk.eliminate_fixed([0, 0])
        assert np.allclose(raw * 2.0 ** e, [0.5, 0.0], atol=1e-7)
        # other outputs: <x|C|00> = (1/2, 1/2, 1/2, -1/2) by the state vector
        for x, ref in [((1, 0), 0.5), ((0, 1), 0.5), ((1, 1), -0.5)]:
            raw, e = p.eliminate_fixed(x)
            assert abs(raw[0] * 2.0 ** e - ref) < 1e-7


def test_amplitudes_report(app_d):
    q = Q()
    c = qi.grid_circuit(4, 4, 12, 0)
    bits = qi.bitstrings(16, 32, 0)
    for executor in EXECS:
        p = q.Plan(q.Model(q.Circuit.grid(4, 4, 12, 0)), batch=32, executor=executor).bind()
        d_bits = torch.from_numpy(bits.astype(np.int64)).cuda()
        d_out = torch.empty(64, dtype=torch.float64, device="cuda")
        r = p.amplitudes_report(d_bits, d_out)
        assert r["status"] == 0 and r["executor"] == executor and r["ms"] > 0
        assert r["slices"] == 1 and r["launches"] >= 1
        assert r["flops"] == p.info.flops_per_slice and r["bytes"] == p.info.bytes_per_slice
        o = d_out.cpu().numpy()
        rel, ab = errors(o[0::2] + 1j * o[1::2], sv.amplitudes(c, bits), 16)
        assert rel < REL_TOL and ab < ABS_TOL

"""ctypes binding of libqgm.so (include/qgm.h): argument marshalling only.

Every step of the amplitude path runs inside the library's CUDA kernels; this
module only converts Python/numpy/torch arguments into the C ABI's plain
pointers and sizes and turns negative status codes into exceptions.  There is
no fallback: if the library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqgm.so")

QGM_OK = 0
ERRORS = {-1: "QGM_ERR_ARG", -2: "QGM_ERR_OOM", -3: "QGM_ERR_CUDA", -4: "QGM_ERR_TIMEOUT",
          -5: "QGM_ERR_NONFINITE", -6: "QGM_ERR_NOGPU"}

ORDER_AUTO, ORDER_MINFILL, ORDER_VERTICAL, ORDER_VERTICAL_T, ORDER_GIVEN = range(5)
OUT_BATCH, OUT_OPEN = 0, 1
EXEC_AUTO, EXEC_STEPWISE, EXEC_RESIDENT, EXEC_COMPILED = 0, 1, 2, 3


class qgm_gate(C.Structure):
    _fields_ = [("kind", C.c_int32), ("cycle", C.c_int32), ("q0", C.c_int32), ("q1", C.c_int32),
                ("theta", C.c_double), ("phi", C.c_double)]


class qgm_model_info(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_vars", C.c_int32), ("n_factors", C.c_int32),
                ("n_nondiag", C.c_int32), ("n_params", C.c_int32)]


class qgm_plan_opts(C.Structure):
    _fields_ = [("order_kind", C.c_int32), ("output_mode", C.c_int32), ("batch", C.c_int64),
                ("mem_budget_bytes", C.c_int64), ("max_fuse", C.c_int32), ("n_order", C.c_int32),
                ("order", C.POINTER(C.c_int32)), ("executor", C.c_int32),
                ("no_gemm", C.c_int32), ("gradients", C.c_int32), ("trees", C.c_int32),
                ("open_mask", C.c_uint64),
                ("resident_chunk", C.c_int32), ("autotune", C.c_int32), ("gemm_precision", C.c_int32),
                ("n_keep", C.c_int32), ("keep_vars", C.POINTER(C.c_int32)), ("tc_convert", C.c_int32)]


class qgm_xeb_result(C.Structure):
    _fields_ = [("cross_entropy", C.c_double), ("alpha", C.c_double), ("mean_Np", C.c_double),
                ("second_moment", C.c_double)]


class qgm_report(C.Structure):
    _fields_ = [("status", C.c_int32), ("executor", C.c_int32), ("ms", C.c_float), ("bytes", C.c_double),
                ("flops", C.c_double), ("slices", C.c_int64), ("launches", C.c_int64)]


class qgm_plan_info(C.Structure):
    _fields_ = [("order_kind", C.c_int32), ("n_free", C.c_int32), ("max_clique", C.c_int32),
                ("n_steps", C.c_int32), ("n_slice_vars", C.c_int32), ("batch_padded", C.c_int32),
                ("n_slices", C.c_int64), ("max_tensor_entries", C.c_int64),
                ("workspace_bytes", C.c_int64), ("arena_bytes", C.c_int64),
                ("bytes_per_slice", C.c_double), ("flops_per_slice", C.c_double),
                ("max_step_bytes", C.c_double), ("n_gemm_steps", C.c_int32), ("n_tile_steps", C.c_int32),
                ("n_nested_steps", C.c_int32), ("n_gemm_tc_steps", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_I64P = C.POINTER(C.c_int64)
_I32P = C.POINTER(C.c_int32)

# name -> (argtypes); every function returns int status unless listed in _VOID
_SIGS = {
    "qgm_circuit_grid": [C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int, C.POINTER(_P)],
    "qgm_circuit_from_gates": [C.c_int, C.POINTER(qgm_gate), C.c_int64, C.POINTER(_P)],
    "qgm_circuit_gates": [_P, C.POINTER(qgm_gate), C.c_int64, _I64P],
    "qgm_circuit_param_gates": [_P, _I32P, C.c_int64, _I64P],
    "qgm_circuit_line_graph_width": [_P, _I32P, _I32P],
    "qgm_plan_kernel_source": [_P, C.c_int32, C.c_int32, C.c_int32, C.c_char_p, C.c_int64, _I64P],
    "qgm_circuit_observable": [_P, C.c_char_p, C.POINTER(_P), C.POINTER(C.c_double), _I32P],
    "qgm_circuit_free": [_P],
    "qgm_build_model": [_P, C.POINTER(_P)],
    "qgm_model_get_info": [_P, C.POINTER(qgm_model_info)],
    "qgm_model_vars": [_P, _I32P, _I32P],
    "qgm_model_factors": [_P, _I32P, _I32P],
    "qgm_model_free": [_P],
    "qgm_plan_order": [_P, C.POINTER(qgm_plan_opts), C.POINTER(_P)],
    "qgm_plan_get_info": [_P, C.POINTER(qgm_plan_info)],
    "qgm_plan_get_order": [_P, _I32P, C.c_int64, _I64P],
    "qgm_plan_get_slice_vars": [_P, _I32P, C.c_int64, _I64P],
    "qgm_plan_get_steps": [_P, _I32P, _I32P, _I32P, _I32P, C.c_int64],
    "qgm_plan_get_step_kernels": [_P, _I32P, C.c_int64],
    "qgm_plan_get_step_cost": [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int64],
    "qgm_plan_get_gemm": [_P, _I32P, C.c_int64, _I64P],
    "qgm_plan_get_tuning": [_P, _I32P, C.POINTER(C.c_float), C.c_int64, _I64P],
    "qgm_plan_set_tuning": [_P, _I32P, C.c_int64],
    "qgm_plan_get_step_inputs": [_P, C.c_int32, _I32P, C.c_int64, _I64P],
    "qgm_plan_profile": [_P, _P, C.c_int64, _P, C.POINTER(C.c_float), _P],
    "qgm_plan_profile_gemm": [_P, _P, C.c_int64, _P, C.POINTER(C.c_float), C.POINTER(C.c_float), _P],
    "qgm_measure_fp32_peak": [C.POINTER(C.c_double), _P],
    "qgm_selftest_wait_timeout": [C.c_int64, C.c_int32, _I32P, _P],
    "qgm_plan_step_stats": [_P, C.POINTER(C.c_uint32), _I32P, C.c_int64, _P],
    "qgm_plan_free": [_P],
    "qgm_plan_bind": [_P, _P, C.c_size_t, _P],
    "qgm_amplitudes": [_P, _P, C.c_int64, _P, _P],
    "qgm_amplitudes_host": [_P, _P, C.c_int64, _P, _P],
    "qgm_eliminate": [_P, _P, _P],
    "qgm_eliminate_fixed": [_P, C.POINTER(C.c_uint8), _P, _I64P, _P],
    "qgm_amplitudes_report": [_P, _P, C.c_int64, _P, C.POINTER(qgm_report), _P],
    "qgm_status": [_P, _P],
    "qgm_plan_get_executor": [_P, _I32P, _I32P, _I64P],
    "qgm_amplitudes_static": [_P, _P, C.c_int64, _P, _P],
    "qgm_amplitude_grad": [_P, _P, C.c_int64, _P, _P, _P, _P],
    "qgm_plan_set_params": [_P, C.POINTER(C.c_double), C.c_int64, _P],
    "qgm_xeb_stats": [_P, C.c_int64, C.c_int, _P, C.POINTER(qgm_xeb_result), _P],
    "qgm_sample_from_set": [_P, C.c_int64, C.c_int64, C.c_uint64, _P, _P, _P],
    "qgm_last_error": [],
}
_VOID = {"qgm_circuit_free", "qgm_model_free", "qgm_plan_free"}

_lib = None


def lib():
    """Load libqgm.so (build it first with paper_1712_05384_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libqgm.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = None if name in _VOID else (C.c_char_p if name == "qgm_last_error" else C.c_int)
        _lib = L
    return _lib


class QgmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def check(rc):
    if rc != QGM_OK:
        raise QgmError(rc, lib().qgm_last_error().decode())
    return rc


def _ptr(x):
    """Device or host address of a torch tensor / numpy array / int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


# ----------------------------------------------------------------- objects
class Circuit:
    def __init__(self, handle):
        self._h = handle

    @classmethod
    def grid(cls, rows, cols, depth, seed=0, param=False):
        h = _P()
        check(lib().qgm_circuit_grid(rows, cols, depth, seed, int(param), C.byref(h)))
        return cls(h)

    @classmethod
    def from_gates(cls, n, gates):
        arr = (qgm_gate * max(len(gates), 1))()
        for i, g in enumerate(gates):
            arr[i] = qgm_gate(int(g.kind), int(g.cycle), int(g.q0), int(g.q1), float(g.theta),
                              float(g.phi))
        h = _P()
        check(lib().qgm_circuit_from_gates(n, arr, len(gates), C.byref(h)))
        return cls(h)

    def gates(self):
        n = C.c_int64()
        check(lib().qgm_circuit_gates(self._h, None, 0, C.byref(n)))
        arr = (qgm_gate * max(n.value, 1))()
        check(lib().qgm_circuit_gates(self._h, arr, n.value, C.byref(n)))
        return [(g.kind, g.cycle, g.q0, g.q1, g.theta, g.phi) for g in arr[: n.value]]

    def param_gates(self):
        n = C.c_int64()
        check(lib().qgm_circuit_param_gates(self._h, None, 0, C.byref(n)))
        a = np.zeros(max(n.value, 1), dtype=np.int32)
        check(lib().qgm_circuit_param_gates(self._h, a.ctypes.data_as(_I32P), n.value, C.byref(n)))
        return a[: n.value]

    def observable(self, pauli: str):
        """(circuit W or None, phase, qubit map) with <0|U^dagger P U|0> =
        phase * <0|W|0> for the Pauli string P (Sec. III, light cone only)."""
        h = _P()
        ph = (C.c_double * 2)()
        qmap = np.zeros(64, dtype=np.int32)
        check(lib().qgm_circuit_observable(self._h, pauli.encode(), C.byref(h), ph,
                                           qmap.ctypes.data_as(_I32P)))
        return (Circuit(h) if h.value else None), complex(ph[0], ph[1]), qmap[: len(pauli)]

    def line_graph_width(self):
        """(segments, max clique) of the min-fill order on the line graph of
        the circuit's tensor network (App. E)."""
        ns, w = C.c_int32(), C.c_int32()
        check(lib().qgm_circuit_line_graph_width(self._h, C.byref(ns), C.byref(w)))
        return ns.value, w.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qgm_circuit_free(self._h)
            self._h = None


class Model:
    def __init__(self, circuit: Circuit):
        self.circuit = circuit
        self._h = _P()
        check(lib().qgm_build_model(circuit._h, C.byref(self._h)))
        self.info = qgm_model_info()
        check(lib().qgm_model_get_info(self._h, C.byref(self.info)))

    def vars(self):
        nv = self.info.n_vars
        q = np.zeros(nv, dtype=np.int32)
        k = np.zeros(nv, dtype=np.int32)
        check(lib().qgm_model_vars(self._h, q.ctypes.data_as(_I32P), k.ctypes.data_as(_I32P)))
        return q, k

    def factors(self):
        nf = self.info.n_factors
        nv = np.zeros(nf, dtype=np.int32)
        sc = np.zeros(2 * nf, dtype=np.int32)
        check(lib().qgm_model_factors(self._h, nv.ctypes.data_as(_I32P), sc.ctypes.data_as(_I32P)))
        return [tuple(sc[2 * f: 2 * f + nv[f]]) for f in range(nf)]

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qgm_model_free(self._h)
            self._h = None


class Plan:
    def __init__(self, model: Model, order_kind=ORDER_AUTO, output_mode=OUT_BATCH, batch=1,
                 mem_budget_bytes=0, max_fuse=0, order=None, executor=EXEC_AUTO,
                 resident_chunk=0, gradients=False, gemm=True, open_mask=0, trees=None,
                 split_bf16=None, precision=None, autotune=False, keep_vars=None, tc_convert=False):
        self.model = model
        o = qgm_plan_opts()
        o.order_kind = order_kind
        o.output_mode = output_mode
        o.batch = batch
        o.mem_budget_bytes = mem_budget_bytes
        o.max_fuse = max_fuse
        o.executor = executor
        o.resident_chunk = resident_chunk
        o.gradients = int(gradients)
        o.no_gemm = 0 if gemm else 1
        o.open_mask = open_mask
        o.trees = 0 if trees is None else (1 if trees else -1)
        # GEMM steps: "fp16" (split FP16 on the tensor cores, the default
        # where eligible), "bf16" (split BF16 on the tensor cores) or "fp32"
        # (FP32 cores); split_bf16=True/False is the same as "bf16"/"fp32"
        if precision is None and split_bf16 is not None:
            precision = "bf16" if split_bf16 else "fp32"
        o.gemm_precision = {None: 0, "fp16": 2, "bf16": 1, "fp32": -1}[precision]
        o.autotune = 1 if autotune else 0
        # folded tensor-core steps convert their batched operand inside the
        # product kernel (else in a split pass of their own)
        o.tc_convert = 1 if tc_convert else 0
        self._keep_buf = None
        if keep_vars is not None and len(keep_vars):
            self._keep_buf = np.ascontiguousarray(keep_vars, dtype=np.int32)
            o.keep_vars = self._keep_buf.ctypes.data_as(_I32P)
            o.n_keep = len(self._keep_buf)
        # amplitudes per bitstring: its open qubits (and kept variables) run
        # over all their values
        self.n_open = (bin(open_mask).count("1") + (0 if self._keep_buf is None else len(self._keep_buf))
                       if output_mode == OUT_BATCH else 0)
        self._order_buf = None
        if order is not None:
            self._order_buf = np.ascontiguousarray(order, dtype=np.int32)
            o.order = self._order_buf.ctypes.data_as(_I32P)
            o.n_order = len(self._order_buf)
            o.order_kind = ORDER_GIVEN
        self._h = _P()
        check(lib().qgm_plan_order(model._h, C.byref(o), C.byref(self._h)))
        self.info = qgm_plan_info()
        check(lib().qgm_plan_get_info(self._h, C.byref(self.info)))
        self.batch = batch
        self.output_mode = output_mode
        self.gradients = bool(gradients)
        self._ws = None

    def order(self):
        n = C.c_int64()
        check(lib().qgm_plan_get_order(self._h, None, 0, C.byref(n)))
        a = np.zeros(max(n.value, 1), dtype=np.int32)
        check(lib().qgm_plan_get_order(self._h, a.ctypes.data_as(_I32P), n.value, C.byref(n)))
        return a[: n.value]

    def slice_vars(self):
        n = C.c_int64()
        check(lib().qgm_plan_get_slice_vars(self._h, None, 0, C.byref(n)))
        a = np.zeros(max(n.value, 1), dtype=np.int32)
        check(lib().qgm_plan_get_slice_vars(self._h, a.ctypes.data_as(_I32P), n.value, C.byref(n)))
        return a[: n.value]

    def steps(self):
        n = self.info.n_steps
        arrs = [np.zeros(max(n, 1), dtype=np.int32) for _ in range(4)]
        check(lib().qgm_plan_get_steps(self._h, *[a.ctypes.data_as(_I32P) for a in arrs], n))
        return {k: a[:n] for k, a in zip(("out_rank", "k", "n_in", "batched"), arrs)}

    def step_kernels(self):
        """Per step: 0 plain, 1 batched, 2 batched with register tile, 3 GEMM,
        4 plain inside a single-CTA run of small steps."""
        n = self.info.n_steps
        a = np.zeros(max(n, 1), dtype=np.int32)
        check(lib().qgm_plan_get_step_kernels(self._h, a.ctypes.data_as(_I32P), n))
        return a[:n]

    def step_costs(self):
        n = self.info.n_steps
        b = np.zeros(max(n, 1))
        f = np.zeros(max(n, 1))
        check(lib().qgm_plan_get_step_cost(self._h, b.ctypes.data_as(C.POINTER(C.c_double)),
                                           f.ctypes.data_as(C.POINTER(C.c_double)), n))
        return b[:n], f[:n]

    def step_inputs(self, step):
        """(union size, k, [(vars as union positions, batched) per input]) of a
        step; union positions < k are the summed variables."""
        n = C.c_int64()
        check(lib().qgm_plan_get_step_inputs(self._h, step, None, 0, C.byref(n)))
        a = np.zeros(max(n.value, 1), dtype=np.int32)
        check(lib().qgm_plan_get_step_inputs(self._h, step, a.ctypes.data_as(_I32P), n.value, C.byref(n)))
        U, k, m = int(a[0]), int(a[1]), int(a[2])
        i, ins = 3, []
        for _ in range(m):
            r, b = int(a[i]), int(a[i + 1])
            ins.append((list(map(int, a[i + 2:i + 2 + r])), b))
            i += 2 + r
        return U, k, ins

    def tuning(self):
        """Autotuner choices after bind: list of dicts (step, nt_cap, T, conv,
        U, ps, ms_rule, ms_best)."""
        n = C.c_int64()
        check(lib().qgm_plan_get_tuning(self._h, None, None, 0, C.byref(n)))
        r = np.zeros(6 * max(n.value, 1), dtype=np.int32)
        m = np.zeros(2 * max(n.value, 1), dtype=np.float32)
        check(lib().qgm_plan_get_tuning(self._h, r.ctypes.data_as(_I32P), m.ctypes.data_as(C.POINTER(C.c_float)),
                                        n.value, C.byref(n)))
        return [{"step": int(r[6 * c]), "nt_cap": int(r[6 * c + 1]), "T": int(r[6 * c + 2]),
                 "conv": int(r[6 * c + 3]), "U": int(r[6 * c + 4]), "ps": int(r[6 * c + 5]),
                 "ms_rule": float(m[2 * c]), "ms_best": float(m[2 * c + 1])}
                for c in range(n.value)]

    def set_tuning(self, choices):
        """Set launch parameters by hand: dicts with step and any of nt_cap,
        T, conv, U, ps (as tuning() returns them)."""
        r = np.zeros(6 * max(len(choices), 1), dtype=np.int32)
        for c, t in enumerate(choices):
            r[6 * c:6 * c + 6] = [t["step"], t.get("nt_cap", 0), t.get("T", 0), t.get("conv", 0), t.get("U", 0),
                                  t.get("ps", 0)]
        check(lib().qgm_plan_set_tuning(self._h, r.ctypes.data_as(_I32P), len(choices)))
        return self

    def gemm_shapes(self):
        """GEMM-shaped steps: list of dicts (step, nm, nn, nk, ns, a_bat,
        b_bat, o_bat, tc, o_bout, in_bout, conv_ok) -- 2^nm x 2^nn outputs,
        2^nk summed entries, for each of the 2^ns shared indices (and batch
        entry when batched); o_bout / in_bout: output / an operand stored with
        the batch entry outermost; conv_ok: a folded tensor-core step (its
        product kernel can convert the batched operand itself)."""
        n = C.c_int64()
        check(lib().qgm_plan_get_gemm(self._h, None, 0, C.byref(n)))
        a = np.zeros(12 * max(n.value, 1), dtype=np.int32)
        check(lib().qgm_plan_get_gemm(self._h, a.ctypes.data_as(_I32P), n.value, C.byref(n)))
        keys = ("step", "nm", "nn", "nk", "ns", "a_bat", "b_bat", "o_bat", "tc", "o_bout", "in_bout", "conv_ok")
        return [dict(zip(keys, map(int, a[12 * c: 12 * c + 12]))) for c in range(n.value)]

    # ------------------------------------------------------------ device
    def bind(self, workspace=None, stream=None):
        """Bind a device workspace (a uint8 torch tensor); allocated here if None."""
        import torch
        if workspace is None:
            workspace = torch.empty(self.info.workspace_bytes + 256, dtype=torch.uint8,
                                    device="cuda")
            off = (-workspace.data_ptr()) % 256
            workspace = workspace[off:]
        check(lib().qgm_plan_bind(self._h, workspace.data_ptr(), workspace.numel(), _stream(stream)))
        self._ws = workspace
        return self

    def amplitudes(self, d_bits, d_out, B=None, stream=None):
        B = d_bits.numel() if B is None else B
        check(lib().qgm_amplitudes(self._h, _ptr(d_bits), B, _ptr(d_out), _stream(stream)))
        return d_out

    def amplitudes_host(self, bits: np.ndarray, stream=None) -> np.ndarray:
        """Amplitudes of host bitstrings: shape (B,), or (B, 2^k) with k open qubits."""
        bits = np.ascontiguousarray(bits, dtype=np.uint64)
        out = np.zeros(2 * (len(bits) << self.n_open), dtype=np.float64)
        check(lib().qgm_amplitudes_host(self._h, bits.ctypes.data, len(bits), out.ctypes.data,
                                        _stream(stream)))
        a = out[0::2] + 1j * out[1::2]
        return a.reshape(len(bits), 1 << self.n_open) if self.n_open else a

    def eliminate(self, d_out, stream=None):
        check(lib().qgm_eliminate(self._h, _ptr(d_out), _stream(stream)))
        return d_out

    def eliminate_fixed(self, x_bits, stream=None):
        """(raw final tensor times the constant, as complex128 of 2^k entries,
        exponent e): the values are raw * 2^e for the output bits x_bits
        (sequence of n 0/1 values, qubit q first)."""
        import torch
        fa = np.ascontiguousarray(x_bits, dtype=np.uint8)
        out = torch.zeros(2 << self.n_open, dtype=torch.float64, device="cuda")
        e = C.c_int64()
        check(lib().qgm_eliminate_fixed(self._h, fa.ctypes.data_as(C.POINTER(C.c_uint8)), _ptr(out), C.byref(e),
                                        _stream(stream)))
        o = out.cpu().numpy()
        return o[0::2] + 1j * o[1::2], e.value

    def amplitudes_report(self, d_bits, d_out, B=None, stream=None):
        """qgm_amplitudes with its report (a dict)."""
        B = d_bits.numel() if B is None else B
        r = qgm_report()
        check(lib().qgm_amplitudes_report(self._h, _ptr(d_bits), B, _ptr(d_out), C.byref(r), _stream(stream)))
        return {k: getattr(r, k) for k, _ in r._fields_}

    def profile(self, d_bits, d_out, B=None, stream=None):
        """Per-kernel milliseconds of one slice: [leaves, step 0..n-1, accumulate]."""
        B = d_bits.numel() if B is None else B
        ms = np.zeros(self.info.n_steps + 2, dtype=np.float32)
        check(lib().qgm_plan_profile(self._h, _ptr(d_bits), B, _ptr(d_out),
                                     ms.ctypes.data_as(C.POINTER(C.c_float)), _stream(stream)))
        return ms

    def profile_gemm(self, d_bits, d_out, B=None, stream=None):
        """Per GEMM step: (split ms, product ms) arrays of one slice."""
        B = d_bits.numel() if B is None else B
        n = self.info.n_gemm_steps
        a = np.zeros(max(n, 1), dtype=np.float32)
        b = np.zeros(max(n, 1), dtype=np.float32)
        check(lib().qgm_plan_profile_gemm(self._h, _ptr(d_bits), B, _ptr(d_out),
                                          a.ctypes.data_as(C.POINTER(C.c_float)),
                                          b.ctypes.data_as(C.POINTER(C.c_float)), _stream(stream)))
        return a[:n], b[:n]

    def step_stats(self, stream=None):
        """(max |value| of each step's scaled output, its exponent) after a run."""
        n = self.info.n_steps
        mb = np.zeros(max(n, 1), dtype=np.uint32)
        ex = np.zeros(max(n, 1), dtype=np.int32)
        check(lib().qgm_plan_step_stats(self._h, mb.ctypes.data_as(C.POINTER(C.c_uint32)), ex.ctypes.data_as(_I32P),
                                        n, _stream(stream)))
        return mb[:n].view(np.float32).copy(), ex[:n]

    def kernel_source(self, chunk=1, part=0, min_blocks=0) -> str:
        """CUDA source of the compiled resident kernel for this plan (no GPU needed)."""
        n = C.c_int64()
        check(lib().qgm_plan_kernel_source(self._h, chunk, part, min_blocks, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value + 1)
        check(lib().qgm_plan_kernel_source(self._h, chunk, part, min_blocks, buf, n.value + 1, C.byref(n)))
        return buf.value.decode()

    def executor(self):
        """(kind, chunk, smem_bytes) of the bound executor."""
        k, c, m = C.c_int32(), C.c_int32(), C.c_int64()
        check(lib().qgm_plan_get_executor(self._h, C.byref(k), C.byref(c), C.byref(m)))
        return k.value, c.value, m.value

    def status(self, stream=None):
        return lib().qgm_status(self._h, _stream(stream))

    def set_params(self, params, stream=None):
        """New (theta, phi) of the RXY gates (flat, 2 per gate) without re-planning."""
        a = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(-1))
        check(lib().qgm_plan_set_params(self._h, a.ctypes.data_as(C.POINTER(C.c_double)), a.size, _stream(stream)))

    def amplitude_grad(self, d_bits, d_dL_dconja, d_grad, d_amp=None, B=None, stream=None):
        B = d_bits.numel() if B is None else B
        check(lib().qgm_amplitude_grad(self._h, _ptr(d_bits), B, _ptr(d_dL_dconja), _ptr(d_grad),
                                       _ptr(d_amp), _stream(stream)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.qgm_plan_free(self._h)
            self._h = None


def measure_fp32_peak(stream=None):
    """FP32 FMA throughput of the current device, TFLOP/s (microbenchmark)."""
    t = C.c_double()
    check(lib().qgm_measure_fp32_peak(C.byref(t), _stream(stream)))
    return t.value


def selftest_wait_timeout(limit_ns, arrive=False, stream=None):
    """Run the kernels' bounded mbarrier wait on a barrier nothing (arrive =
    False) or the waiting thread itself (True) arrives at; returns the status
    the kernel wrote (QGM_ERR_TIMEOUT or 0)."""
    st = C.c_int32(1)
    check(lib().qgm_selftest_wait_timeout(int(limit_ns), 1 if arrive else 0, C.byref(st), _stream(stream)))
    return st.value


# ---------------------------------------------------------------- App. B, C
def xeb_stats(d_amps, B, n_qubits, d_scratch, stream=None):
    """Cross-entropy statistics of B device amplitudes (see qgm_xeb_stats)."""
    r = qgm_xeb_result()
    check(lib().qgm_xeb_stats(_ptr(d_amps), B, n_qubits, _ptr(d_scratch), C.byref(r), _stream(stream)))
    return {k: getattr(r, k) for k, _ in r._fields_}


def sample_from_set(d_amps, t, m, seed, d_scratch, d_idx, stream=None):
    """m indices drawn from the t amplitudes with p/sum p (see qgm_sample_from_set)."""
    check(lib().qgm_sample_from_set(_ptr(d_amps), t, m, seed, _ptr(d_scratch), _ptr(d_idx),
                                    _stream(stream)))
    return d_idx

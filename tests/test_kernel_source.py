"""The compiled resident kernel's source compiles for sm_103a on the host
(NVRTC, no GPU needed): whole passes for chunks of 1, 2 and 4 bitstrings,
the batched and bitstring-independent parts, nested steps, contraction
trees and a parametrised circuit.  Skipped where NVRTC is not installed."""
import ctypes as C
import os

import pytest

import paper_1712_05384_gb300 as Q

NVRTC_NAMES = ["libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"]


def nvrtc():
    for name in NVRTC_NAMES:
        try:
            return C.CDLL(name)
        except OSError:
            continue
    pytest.skip("NVRTC not installed")


def compile_source(src: str):
    lib = nvrtc()
    prog = C.c_void_p()
    assert lib.nvrtcCreateProgram(C.byref(prog), src.encode(), b"k.cu", 0, None, None) == 0
    opts = [b"--gpu-architecture=sm_103a", b"-std=c++17", b"-default-device"]
    arr = (C.c_char_p * len(opts))(*opts)
    rc = lib.nvrtcCompileProgram(prog, len(opts), arr)
    n = C.c_size_t()
    lib.nvrtcGetProgramLogSize(prog, C.byref(n))
    log = C.create_string_buffer(n.value + 1)
    lib.nvrtcGetProgramLog(prog, log)
    size = C.c_size_t()
    lib.nvrtcGetCUBINSize(prog, C.byref(size))
    lib.nvrtcDestroyProgram(C.byref(prog))
    return rc, log.value.decode(errors="replace"), size.value


@pytest.mark.parametrize("case", ["4x4_d12", "4x4_d12_chunk2", "4x4_d12_chunk4", "3x4_d14_param",
                                  "4x4_d14_trees", "5x5_d20_parts"])
def test_generated_kernel_compiles(case):
    grid = {"4x4_d12": (4, 4, 12, False), "4x4_d12_chunk2": (4, 4, 12, False),
            "4x4_d12_chunk4": (4, 4, 12, False), "3x4_d14_param": (3, 4, 14, True),
            "4x4_d14_trees": (4, 4, 14, False), "5x5_d20_parts": (5, 5, 20, False)}[case]
    r, c, d, param = grid
    p = Q.Plan(Q.Model(Q.Circuit.grid(r, c, d, 0, param)), batch=64, trees=case.endswith("trees"))
    chunk = 2 if case.endswith("chunk2") else 4 if case.endswith("chunk4") else 1
    parts = [1, 2] if case.endswith("parts") else [0]
    for part in parts:
        src = p.kernel_source(chunk, part)
        assert "extern \"C\" __global__" in src
        rc, log, cubin = compile_source(src)
        assert rc == 0, log[-2000:]
        assert cubin > 0


def test_kernel_source_errors():
    p = Q.Plan(Q.Model(Q.Circuit.grid(3, 3, 8, 0)), batch=8)
    with pytest.raises(Q.QgmError):
        p.kernel_source(16)          # no layout with 16 bitstrings per CTA
    with pytest.raises(Q.QgmError):
        p.kernel_source(1, part=3)

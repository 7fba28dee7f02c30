"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/ftgcr.h declares; the binding fails loudly when the library is
missing (no CPU fallback).  No compute calls: these run without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2103_07210_gb300 import ftgcr

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ftgcr.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ftgcr_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_binding_exports():
    assert sorted(ftgcr.EXPORTS) == declared_functions()


def test_library_builds_and_exports_every_declared_symbol():
    path = ftgcr.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [f for f in declared_functions() if f not in syms]
    assert not missing, missing
    L = ctypes.CDLL(path)
    for f in declared_functions():
        assert hasattr(L, f)


def test_build_flags_target_sm_103a_only():
    assert "arch=compute_103a,code=sm_103a" in ftgcr.NVCC_FLAGS
    assert "--fmad=false" in ftgcr.NVCC_FLAGS


def test_error_strings_without_gpu():
    L = ftgcr.lib()
    assert L.ftgcr_error_string(0) == b"ok"
    assert b"timed out" in L.ftgcr_error_string(-4)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(ftgcr, "_lib", None)
    monkeypatch.setattr(ftgcr, "LIB_PATH", str(tmp_path / "nope" / "libftgcr.so"))

    def no_build(*a, **k):
        raise RuntimeError("build disabled")

    monkeypatch.setattr(ftgcr, "build", no_build)
    with pytest.raises(Exception):
        ftgcr.lib()


def test_server_refuses_bad_arguments_and_a_missing_gpu_without_crashing():
    L = ftgcr.lib()
    srv = ctypes.c_void_p()
    assert L.ftgcr_server_create(0, 0, 8, ctypes.byref(srv)) == ftgcr.ERR_ARG  # no slots
    assert L.ftgcr_server_create(0, 1025, 8, ctypes.byref(srv)) == ftgcr.ERR_ARG  # above the table limit
    assert L.ftgcr_server_create(-1, 4, 8, ctypes.byref(srv)) == ftgcr.ERR_ARG
    assert L.ftgcr_server_create(0, 4, 0, ctypes.byref(srv)) == ftgcr.ERR_ARG
    import torch
    if not torch.cuda.is_available():
        assert L.ftgcr_server_create(0, 4, 8, ctypes.byref(srv)) == ftgcr.ERR_CUDA
        assert srv.value is None


def test_round_layout_flags_are_validated_before_any_device_call():
    import numpy as np

    L = ftgcr.lib()
    D = np.ones((8, 16))
    h = ctypes.c_void_p()
    c = ftgcr.Coeffs(D.ctypes.data, 0)
    bad = [ftgcr._grid(16, 8, 1.0, "mixed", "line", 0, 0, 0.0, 0, rounds="split"),
           ftgcr._grid(16, 8, 1.0, "fp64", "line", 0, 0, 0.0, 0, rounds="split"),  # FP64 has no split rounds
           ftgcr._grid(16, 8, 1.0, "mixed", "jacobi", 0, 0, 0.0, 0, rounds="split"),
           ftgcr._grid(16, 8, 1.0, "fp64", "line", 0, 0, 0.0, 0, rounds="streamed"),  # mixed path only
           ftgcr._grid(16, 8, 1.0, "mixed", "identity", 0, 0, 0.0, 0, rounds="streamed"),
           ftgcr._grid(16, 8, 1.0, "mixed", "line", 0, 0, 0.0, 0, rounds="streamed"),
           ftgcr._grid(16, 8, 1.0, "mixed", "line", 0, 0, 0.0, 0, oracle_order=True),  # FP64 path only
           ftgcr._grid(16, 8, 1.0, "mixed", "jacobi", 0, 0, 0.0, 0, oracle_order=True)]
    bad[0].flags |= ftgcr.FLAG_FUSED_ROUNDS  # both layouts at once
    bad[5].flags |= ftgcr.FLAG_SPLIT_ROUNDS
    for g in bad:
        assert L.ftgcr_create(ctypes.byref(g), ctypes.byref(c), 4, 1e-10, ctypes.byref(h)) == ftgcr.ERR_ARG
    unknown = ftgcr._grid(16, 8, 1.0, "mixed", "line", 0, 0, 0.0, 0)
    unknown.flags = 64
    assert L.ftgcr_create(ctypes.byref(unknown), ctypes.byref(c), 4, 1e-10, ctypes.byref(h)) == ftgcr.ERR_ARG


def test_tune_refuses_bad_arguments_before_any_device_call():
    import numpy as np

    L = ftgcr.lib()
    D = np.ones((8, 16))
    c = ftgcr.Coeffs(D.ctypes.data, 0)
    t = ftgcr.Tuning()
    g = ftgcr._grid(16, 8, 1.0, "mixed", "line", 0, 0, 0.0, 0)
    for conc in (0, ftgcr.TUNE_MAX_CONCURRENCY + 1):
        assert L.ftgcr_tune(ctypes.byref(g), ctypes.byref(c), 4, 1e-10, conc, ctypes.byref(t)) == ftgcr.ERR_ARG
    fixed = ftgcr._grid(16, 8, 1.0, "mixed", "line", 0, 4, 0.0, 0)  # tiles given: the tuner chooses them
    assert L.ftgcr_tune(ctypes.byref(fixed), ctypes.byref(c), 4, 1e-10, 1, ctypes.byref(t)) == ftgcr.ERR_ARG
    forced = ftgcr._grid(16, 8, 1.0, "mixed", "line", 0, 0, 0.0, 0, rounds="split")
    assert L.ftgcr_tune(ctypes.byref(forced), ctypes.byref(c), 4, 1e-10, 1, ctypes.byref(t)) == ftgcr.ERR_ARG
    import torch
    if not torch.cuda.is_available():
        assert L.ftgcr_tune(ctypes.byref(g), ctypes.byref(c), 4, 1e-10, 1, ctypes.byref(t)) == ftgcr.ERR_CUDA


def test_fma_rate_probe_refuses_bad_arguments_before_any_device_call():
    L = ftgcr.lib()
    t = ctypes.c_double(1.0)
    for iters in (0, -1, (1 << 24) + 1):
        assert L.ftgcr_fp64_fma_rate(iters, ctypes.byref(t), None) == ftgcr.ERR_ARG
    assert L.ftgcr_fp64_fma_rate(16, None, None) == ftgcr.ERR_ARG
    import torch
    if not torch.cuda.is_available():
        assert L.ftgcr_fp64_fma_rate(16, ctypes.byref(t), None) == ftgcr.ERR_CUDA and t.value == 0.0


def test_host_async_solve_refuses_null_arguments_before_any_device_call():
    L = ftgcr.lib()
    buf = (ctypes.c_double * 4)()
    assert L.ftgcr_solve_host_async(None, buf, buf, None, None) == ftgcr.ERR_ARG

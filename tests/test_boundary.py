"""The C ABI without a GPU: libpdas builds, loads, exports every entry point
that include/*.h declares (as unmangled C symbols), and rejects bad
arguments on the host before touching the device."""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(pdas_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1502_03543_gb300 import build as B
    path = B.build()
    return ctypes.CDLL(path), path


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pdas_create", "pdas_solve", "pdas_step", "pdas_backward", "pdas_destroy", "pdas_status_str",
                     "pdas_last_error_index"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    handle, path = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in declared_functions() if n not in exported or not hasattr(handle, n)]
    assert not missing, missing


def test_host_side_validation_without_gpu(lib):
    from paper_1502_03543_gb300 import _native as N
    L = N.lib()
    o = N.Options()
    L.pdas_default_options(ctypes.byref(o))
    assert o.max_iter == 500 and o.refine_tol == 1e-14 and o.dspread_refactor == 0.0 and o.form == N.FP64
    assert o.refine_be == 1e-14 and o.drop_tol == 1e-10 and o.drop_keep == 1.25 and o.refine_max == 40
    assert o.exact_passes == 0 and o.infeasible == 0
    h = ctypes.c_void_p()
    # m < n and m >= 1 (Section I)
    assert L.pdas_create(10, 10, ctypes.byref(o), ctypes.byref(h)) == N.ERR_ARG
    assert L.pdas_create(0, 10, ctypes.byref(o), ctypes.byref(h)) == N.ERR_ARG
    assert L.pdas_create(12, 5, ctypes.byref(o), ctypes.byref(h)) == N.ERR_ARG
    assert not h.value
    bad = N.Options.from_buffer_copy(o)
    bad.form = 9
    assert L.pdas_create(3, 5, ctypes.byref(bad), ctypes.byref(h)) == N.ERR_ARG
    bad = N.Options.from_buffer_copy(o)
    bad.exact_passes = 2
    assert L.pdas_create(3, 5, ctypes.byref(bad), ctypes.byref(h)) == N.ERR_ARG
    bad = N.Options.from_buffer_copy(o)
    bad.infeasible = 2
    assert L.pdas_create(3, 5, ctypes.byref(bad), ctypes.byref(h)) == N.ERR_ARG
    bad = N.Options.from_buffer_copy(o)
    bad.refine_tol = -1.0
    assert L.pdas_create(3, 5, ctypes.byref(bad), ctypes.byref(h)) == N.ERR_ARG
    # BF16 operands need BF16 storage
    bad = N.Options.from_buffer_copy(o)
    bad.form, bad.a_dtype = N.BF16_IR, N.A_F64
    assert L.pdas_create(3, 5, ctypes.byref(bad), ctypes.byref(h)) == N.ERR_UNSUPPORTED
    # TF32 operands: FP64 or FP32 storage, one product or TF32 x 3
    bad = N.Options.from_buffer_copy(o)
    bad.form, bad.a_dtype = N.TF32_IR, N.A_BF16
    assert L.pdas_create(3, 5, ctypes.byref(bad), ctypes.byref(h)) == N.ERR_UNSUPPORTED
    bad = N.Options.from_buffer_copy(o)
    bad.form, bad.splits = N.TF32_IR, 2
    assert L.pdas_create(3, 5, ctypes.byref(bad), ctypes.byref(h)) == N.ERR_UNSUPPORTED
    assert not h.value
    # null handle / pointers
    assert L.pdas_step(None, None, None, None, None, None, None, 0.5, None) == N.ERR_ARG
    assert L.pdas_solve(None, None, None, None, None, None, None, 0.5, 1e-8, None, None) == N.ERR_ARG
    assert L.pdas_last_error_index(None) == -1
    L.pdas_destroy(None)
    for code in range(-7, 6):
        assert len(N.status_str(code)) > 0


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1502_03543_gb300 import _native as N
    monkeypatch.setattr(N, "_lib", None)
    monkeypatch.setattr(N, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        N.lib()


def test_binding_refuses_host_tensors():
    """No CPU fallback: the binding accepts device tensors only, and checks
    dtype, size and contiguity before anything reaches the library."""
    import torch
    from paper_1502_03543_gb300 import _ptr
    with pytest.raises(TypeError, match="CUDA tensor"):
        _ptr(torch.zeros(4, dtype=torch.float64), torch.float64, 4, "x")
    with pytest.raises(TypeError, match="CUDA tensor"):
        _ptr([0.0] * 4, torch.float64, 4, "x")

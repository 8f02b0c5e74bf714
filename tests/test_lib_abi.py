"""The C-ABI library builds, loads and exports every symbol include/pat.h declares (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import importlib
    b = importlib.import_module("paper_1605_00133_gb300.build")
    b.build()
    from paper_1605_00133_gb300 import _lib
    return _lib.load()


def declared_functions(header="pat.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pat_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("pat_create_grid", "pat_forward", "pat_adjoint", "pat_destroy_grid", "pat_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1605_00133_gb300 import _lib
    names = declared_functions()
    assert sorted(_lib.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n
    assert lib.pat_version().startswith(b"libpat")
    unet = declared_functions("pat_unet.h")
    assert sorted(_lib.UNET_EXPORTS) == unet
    for n in unet:
        assert hasattr(lib, n), n
    assert sorted(os.listdir(os.path.join(ROOT, "include"))) == ["pat.h", "pat_unet.h"]


def _desc(**kw):
    from paper_1605_00133_gb300 import _lib
    d = dict(nz=16, ny=16, nx=16, dx=1e-4, c=1500.0, rho0=1.0, cfl=0.3, dt=0.0, T=4, pml_size=2,
             pml_alpha=2.0, sensor_z=-1, batch=1)
    d.update(kw)
    return _lib.GridDesc(**d)


@pytest.mark.parametrize("bad", [dict(nx=12), dict(nz=512), dict(T=0), dict(batch=0), dict(pml_size=8),
                                 dict(sensor_z=16), dict(dx=0.0), dict(cfl=0.0)])
def test_invalid_descriptors_are_rejected_before_any_device_call(lib, bad):
    from paper_1605_00133_gb300 import _lib
    d = _desc(**bad)
    s = _lib.SamplingDesc(0, 0, None, None, None)
    h = ctypes.c_void_p()
    st = lib.pat_create_grid(ctypes.byref(d), ctypes.byref(s), ctypes.byref(h))
    assert st == 1 and not h.value
    assert len(lib.pat_last_error()) > 0


def test_invalid_index_sets_are_rejected(lib):
    from paper_1605_00133_gb300 import _lib
    d = _desc()
    h = ctypes.c_void_p()
    dup = np.array([3, 3], np.int32)
    s = _lib.SamplingDesc(1, 2, dup.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), None, None)
    assert lib.pat_create_grid(ctypes.byref(d), ctypes.byref(s), ctypes.byref(h)) == 1
    assert b"duplicate" in lib.pat_last_error()
    perm = np.zeros(256, np.int32)
    rows = np.array([1], np.int32)
    s = _lib.SamplingDesc(2, 1, None, perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                          rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    assert lib.pat_create_grid(ctypes.byref(d), ctypes.byref(s), ctypes.byref(h)) == 1
    assert b"permutation" in lib.pat_last_error()
    big = _desc(ny=256, nx=256)
    perm = np.arange(65536, dtype=np.int32)
    s = _lib.SamplingDesc(2, 1, None, perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                          rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    assert lib.pat_create_grid(ctypes.byref(big), ctypes.byref(s), ctypes.byref(h)) == 6


def test_null_arguments(lib):
    assert lib.pat_forward(None, None, None, None) == 1
    assert lib.pat_adjoint(None, None, None, None) == 1
    assert lib.pat_sample(None, None, None, 1, None) == 1
    lib.pat_destroy_grid(None)


def test_no_gpu_means_an_error_not_a_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1605_00133_gb300 import _lib
    d = _desc()
    s = _lib.SamplingDesc(0, 0, None, None, None)
    h = ctypes.c_void_p()
    assert lib.pat_create_grid(ctypes.byref(d), ctypes.byref(s), ctypes.byref(h)) == 2
    with pytest.raises(RuntimeError):
        from paper_1605_00133_gb300 import PatOperator, presets
        PatOperator(presets.Grid(16, 16, 16, T=4, pml_size=2), presets.Sampling(0, 256))


def test_workspace_cap_returns_oom_before_any_device_call(lib):
    """pat_set_workspace_limit: a grid whose workspace exceeds the cap is refused with PAT_ERR_OOM
    from the host-side size computation alone, whether or not a GPU is present."""
    from paper_1605_00133_gb300 import _lib
    d = _desc(nz=64, ny=128, nx=128, T=400, pml_size=10)
    s = _lib.SamplingDesc(0, 0, None, None, None)
    h = ctypes.c_void_p()
    try:
        assert lib.pat_set_workspace_limit(-1) == 1
        assert lib.pat_set_workspace_limit(10 << 20) == 0
        assert lib.pat_create_grid(ctypes.byref(d), ctypes.byref(s), ctypes.byref(h)) == 3
        assert not h.value
        assert b"pat_set_workspace_limit" in lib.pat_last_error()
    finally:
        assert lib.pat_set_workspace_limit(0) == 0


def test_fault_hook_checks_its_arguments(lib):
    assert lib.pat_debug_copy_fault(None, 2, 4) == 1
    assert lib.pat_device_status(None, None) == 1

"""The C-ABI library loads and exports what include/fft3d.h declares; host-side
argument checks answer before any CUDA call.  No GPU needed."""
import ctypes
import os
import re

import pytest

import paper_2202_12756_gb300 as fft3d
from paper_2202_12756_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fft3d.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return fft3d.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fft3d_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_binding_names():
    assert set(declared_functions()) == set(fft3d.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_is_cuda_code_for_sm103a():
    # the build targets sm_103a only
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


def test_strerror(lib):
    assert fft3d.fft3d_strerror(fft3d.FFT3D_OK) == "ok"
    assert "size" in fft3d.fft3d_strerror(fft3d.FFT3D_ERR_SIZE)
    assert fft3d.fft3d_strerror(12345) == "unknown status"


POW2 = [2 ** k for k in range(12)]
POW2X3 = [3 * 2 ** k for k in range(10)]


def test_supported_lengths(lib):
    for n in range(0, 4100):
        want01 = n in POW2 or n in POW2X3
        assert fft3d.fft3d_supported_length(n, 0) == want01, n
        assert fft3d.fft3d_supported_length(n, 1) == want01, n
        want2 = n % 2 == 0 and n >= 2 and ((n // 2) in POW2[:11] or (n // 2) in POW2X3[:9])
        assert fft3d.fft3d_supported_length(n, 2) == want2, n
    assert not fft3d.fft3d_supported_length(8, 3)
    assert not fft3d.fft3d_supported_length(-4, 0)


def test_plan_create_rejects_before_touching_cuda(lib):
    h = ctypes.c_void_p(1234)
    assert lib.fft3d_plan_create(ctypes.byref(h), 8, 8, 7, fft3d.FFT3D_F32) == fft3d.FFT3D_ERR_SIZE
    assert h.value is None
    assert lib.fft3d_plan_create(ctypes.byref(h), 5, 8, 8, fft3d.FFT3D_F32) == fft3d.FFT3D_ERR_SIZE
    assert lib.fft3d_plan_create(ctypes.byref(h), 8, 4096, 8, fft3d.FFT3D_F64) == fft3d.FFT3D_ERR_SIZE
    assert lib.fft3d_plan_create(ctypes.byref(h), 8, 8, 4096, fft3d.FFT3D_F64) == fft3d.FFT3D_ERR_SIZE
    assert lib.fft3d_plan_create(ctypes.byref(h), 8, 8, 8, 7) == fft3d.FFT3D_ERR_DTYPE
    assert lib.fft3d_plan_create(None, 8, 8, 8, 0) == fft3d.FFT3D_ERR_NULL
    with pytest.raises(fft3d.FFT3DError) as e:
        fft3d.fft3d_plan_create(6, 10, 8, fft3d.FFT3D_F32)
    assert e.value.status == fft3d.FFT3D_ERR_SIZE


def test_batched_plan_create_rejects_before_touching_cuda(lib):
    h = ctypes.c_void_p(1234)
    create = lib.fft3d_plan_create_batched
    for batch in (0, -3, (1 << 31) // (1024 * 1024) + 1):
        assert create(ctypes.byref(h), batch, 1024, 1024, 64, fft3d.FFT3D_F32) == fft3d.FFT3D_ERR_SIZE
        assert h.value is None
    assert create(ctypes.byref(h), 2, 8, 8, 7, fft3d.FFT3D_F32) == fft3d.FFT3D_ERR_SIZE
    assert create(ctypes.byref(h), 2, 8, 8, 8, 9) == fft3d.FFT3D_ERR_DTYPE
    assert create(None, 2, 8, 8, 8, 0) == fft3d.FFT3D_ERR_NULL


def test_null_plan_calls(lib):
    assert lib.fft3d_plan_destroy(None) == fft3d.FFT3D_OK
    for f in ("fft3d_exec_r2c", "fft3d_exec_c2r", "fft3d_exec_r2c_adjoint", "fft3d_exec_c2r_adjoint"):
        assert getattr(lib, f)(None, 16, 16, None) == fft3d.FFT3D_ERR_NULL
    assert lib.fft3d_plan_set_profiling(None, 1) == fft3d.FFT3D_ERR_NULL
    assert fft3d.fft3d_plan_last_error(None) == ""


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(fft3d.FFT3DError):
        fft3d.load_library(str(tmp_path / "nope.so"))


def test_diagnostics_reject_null_before_touching_cuda(lib):
    D = ctypes.POINTER(ctypes.c_double)
    assert lib.fft3d_noalloc_status(None) == fft3d.FFT3D_ERR_NULL
    assert lib.fft3d_measure_fp64_peak(D(), D(), D()) == fft3d.FFT3D_ERR_NULL

"""FP64 CPU oracle for the 3D R2C / C2R FFT (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The CUDA library never does, and the two
share no code: this wrapper loads ``oracle.c`` compiled with gcc.

Functions follow Sec. 2 of arXiv 2202.12756:
  * ``rfft3``  -- Eq. 1, unnormalised, half spectrum k2 = 0..N2/2 (Eqs. 3-4).
  * ``irfft3`` -- Eq. 2 on the Hermitian extension, times 1/(N0 N1 N2)
                  (the normalisation step of Sec. 4).
  * ``rfft3_adjoint`` / ``irfft3_adjoint`` -- closed-form adjoints derived
                  from those definitions (used for gradient checks).
  * ``fft1d``  -- the oracle's own 1D C2C, exposed for per-line checks.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

# -fcx-limited-range: textbook complex multiply (no C99 inf/nan recovery
# path); -ffp-contract=off: the same rounding on x86 and aarch64.
CFLAGS = ["-O2", "-std=gnu99", "-fPIC", "-shared", "-fopenmp",
          "-fcx-limited-range", "-ffp-contract=off"]

_lock = threading.Lock()
_lib = None


def build(src=_SRC, out=_LIB_PATH, extra_flags=()):
    """Compile ``src`` into the shared library ``out`` with gcc."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", *CFLAGS, *extra_flags, src, "-o", out, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def _declare(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    L = ctypes.c_long
    lib.oracle_fft1d.argtypes = [dp, L, L, ctypes.c_int]
    lib.oracle_rfft3.argtypes = [dp, L, L, L, dp]
    lib.oracle_irfft3.argtypes = [dp, L, L, L, dp]
    lib.oracle_rfft3_adjoint.argtypes = [dp, L, L, L, dp]
    lib.oracle_irfft3_adjoint.argtypes = [dp, L, L, L, dp]
    for f in ("oracle_fft1d", "oracle_rfft3", "oracle_irfft3",
              "oracle_rfft3_adjoint", "oracle_irfft3_adjoint", "oracle_num_threads"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


def load(path=None):
    """Load (building first if needed) the oracle library; returns a handle."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            if (not os.path.exists(_LIB_PATH)
                    or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
                build()
            _lib = _declare(ctypes.CDLL(_LIB_PATH))
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, name):
    if rc != 0:
        raise RuntimeError(f"{name} failed with status {rc}")


def num_threads(lib=None):
    return (lib or load()).oracle_num_threads()


def fft1d(x, sign=-1, lib=None):
    """Unnormalised C2C along the last axis: sum_j x[j] exp(sign 2 pi i j k / n)."""
    lib = lib or load()
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    n = a.shape[-1]
    _check(lib.oracle_fft1d(_ptr(a), n, a.size // max(n, 1), sign), "oracle_fft1d")
    return a


def rfft3(f, lib=None):
    """f: real [N0][N1][N2] -> complex [N0][N1][N2//2+1] (Eq. 1, unnormalised)."""
    lib = lib or load()
    f = np.ascontiguousarray(f, dtype=np.float64)
    n0, n1, n2 = f.shape
    F = np.empty((n0, n1, n2 // 2 + 1), dtype=np.complex128)
    _check(lib.oracle_rfft3(_ptr(f), n0, n1, n2, _ptr(F)), "oracle_rfft3")
    return F


def irfft3(F, shape, lib=None):
    """F: complex [N0][N1][N2//2+1] -> real [N0][N1][N2] (Eq. 2, x 1/(N0 N1 N2))."""
    lib = lib or load()
    F = np.ascontiguousarray(F, dtype=np.complex128)
    n0, n1, n2 = shape
    assert F.shape == (n0, n1, n2 // 2 + 1), (F.shape, shape)
    f = np.empty((n0, n1, n2), dtype=np.float64)
    _check(lib.oracle_irfft3(_ptr(F), n0, n1, n2, _ptr(f)), "oracle_irfft3")
    return f


def rfft3_adjoint(G, shape, lib=None):
    """Adjoint of rfft3: g[j] = Re sum_{k in half} G[k] exp(+2 pi i k.j/N)."""
    lib = lib or load()
    G = np.ascontiguousarray(G, dtype=np.complex128)
    n0, n1, n2 = shape
    assert G.shape == (n0, n1, n2 // 2 + 1)
    g = np.empty((n0, n1, n2), dtype=np.float64)
    _check(lib.oracle_rfft3_adjoint(_ptr(G), n0, n1, n2, _ptr(g)), "oracle_rfft3_adjoint")
    return g


def irfft3_adjoint(g, lib=None):
    """Adjoint of irfft3: G[k] = c(k2)/(N0 N1 N2) * sum_j g[j] exp(-2 pi i k.j/N)."""
    lib = lib or load()
    g = np.ascontiguousarray(g, dtype=np.float64)
    n0, n1, n2 = g.shape
    G = np.empty((n0, n1, n2 // 2 + 1), dtype=np.complex128)
    _check(lib.oracle_irfft3_adjoint(_ptr(g), n0, n1, n2, _ptr(G)), "oracle_irfft3_adjoint")
    return G

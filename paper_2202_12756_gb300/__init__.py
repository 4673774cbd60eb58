"""GB300-native single-GPU 3D real FFT (R2C forward, normalised C2R inverse).

The compute path is the CUDA library ``libfft3d.so`` (sources in ``csrc/``,
C ABI in ``include/fft3d.h``).  This module only marshals arguments:

* ``fft3d_*`` functions mirror the C entry points one to one (plain integer
  handles and device pointers);
* ``Plan`` / ``rfft3`` / ``irfft3`` wrap them for torch CUDA tensors, using
  torch only for device memory and the current stream; ``rfft3`` and
  ``irfft3`` are autograd functions whose backward passes call the library's
  adjoint entry points.

There is no fallback: if the library is missing or a call fails, an
``FFT3DError`` is raised.

The transform is the one of Sec. 2 of arXiv 2202.12756 (Eq. 1 forward,
unnormalised; Eq. 2 inverse with the 1/N^3 normalisation step; half spectrum
k2 = 0..N2/2 per Eqs. 3-4), computed with the single-GPU pass structure
described in ``include/fft3d.h``.
"""
import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfft3d.so")

FFT3D_F32 = 0
FFT3D_F64 = 1

FFT3D_OK = 0
FFT3D_ERR_SIZE = 1
FFT3D_ERR_DTYPE = 2
FFT3D_ERR_NULL = 3
FFT3D_ERR_ALIGN = 4
FFT3D_ERR_ALLOC = 5
FFT3D_ERR_CUDA = 6
FFT3D_ERR_LAYOUT = 7
FFT3D_ERR_DEVICE = 8
FFT3D_ERR_ARG = 9

# every symbol the C header declares
EXPORTED = (
    "fft3d_plan_create", "fft3d_plan_destroy", "fft3d_exec_r2c", "fft3d_exec_c2r",
    "fft3d_exec_r2c_adjoint", "fft3d_exec_c2r_adjoint", "fft3d_strerror",
    "fft3d_plan_last_error", "fft3d_supported_length", "fft3d_plan_set_profiling",
    "fft3d_plan_profile_read", "fft3d_plan_launch_count", "fft3d_exec_c2r_noalloc",
    "fft3d_plan_status", "fft3d_plan_set_debug", "fft3d_plan_info", "fft3d_plan_set_fused",
    "fft3d_exec_c2r_overwrite", "fft3d_plan_create_batched", "fft3d_noalloc_status",
    "fft3d_measure_fp64_peak",
)


class FFT3DError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        msg = f"{where}: {_strerror_raw(status)} (status {status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("bytes_per_launch", ctypes.c_double)]


_lib = None
_lib_lock = threading.RLock()


def _declare(lib):
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    lib.fft3d_plan_create.argtypes = [ctypes.POINTER(P), I64, I64, I64, ctypes.c_int]
    lib.fft3d_plan_create_batched.argtypes = [ctypes.POINTER(P), I64, I64, I64, I64, ctypes.c_int]
    lib.fft3d_plan_destroy.argtypes = [P]
    for f in ("fft3d_exec_r2c", "fft3d_exec_c2r", "fft3d_exec_r2c_adjoint", "fft3d_exec_c2r_adjoint",
              "fft3d_exec_c2r_overwrite"):
        getattr(lib, f).argtypes = [P, P, P, P]
    lib.fft3d_strerror.argtypes = [ctypes.c_int]
    lib.fft3d_strerror.restype = ctypes.c_char_p
    lib.fft3d_plan_last_error.argtypes = [P]
    lib.fft3d_plan_last_error.restype = ctypes.c_char_p
    lib.fft3d_supported_length.argtypes = [I64, ctypes.c_int]
    lib.fft3d_plan_set_profiling.argtypes = [P, ctypes.c_int]
    lib.fft3d_plan_profile_read.argtypes = [P, ctypes.POINTER(KernelStat), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]
    lib.fft3d_plan_launch_count.argtypes = [P, ctypes.POINTER(I64)]
    lib.fft3d_exec_c2r_noalloc.argtypes = [P, P, I64, I64, I64, ctypes.c_int, P]
    lib.fft3d_plan_status.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
    lib.fft3d_plan_set_debug.argtypes = [P, ctypes.c_int, I64]
    lib.fft3d_plan_info.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
    lib.fft3d_plan_set_fused.argtypes = [P, ctypes.c_int]
    lib.fft3d_noalloc_status.argtypes = [ctypes.POINTER(ctypes.c_int)]
    D = ctypes.POINTER(ctypes.c_double)
    lib.fft3d_measure_fp64_peak.argtypes = [D, D, D]
    return lib


def load_library(path=LIB_PATH):
    """Load libfft3d.so (built by ``__graft_entry__.build()`` or ``_build.py``)."""
    global _lib
    with _lib_lock:
        if _lib is None or path != LIB_PATH:
            if not os.path.exists(path):
                raise FFT3DError(FFT3D_ERR_CUDA, "load_library",
                                 f"{path} is missing; build it with paper_2202_12756_gb300/_build.py")
            lib = _declare(ctypes.CDLL(path))
            if path != LIB_PATH:
                return lib
            _lib = lib
    return _lib


_STATUS_TEXT = {
    FFT3D_OK: "ok", FFT3D_ERR_SIZE: "unsupported transform size", FFT3D_ERR_DTYPE: "unsupported dtype",
    FFT3D_ERR_NULL: "null pointer argument",
    FFT3D_ERR_ALIGN: "data pointer not aligned to one complex element",
    FFT3D_ERR_ALLOC: "allocation failed", FFT3D_ERR_CUDA: "CUDA error",
    FFT3D_ERR_LAYOUT: "input and output overlap without being identical",
    FFT3D_ERR_DEVICE: "current device is not the plan's device", FFT3D_ERR_ARG: "invalid argument",
}


def _strerror_raw(status):
    # same text as fft3d_strerror, without needing the library (so that a
    # missing library can still be reported)
    return _STATUS_TEXT.get(int(status), "unknown status")


def _check(rc, where, plan=None):
    if rc != FFT3D_OK:
        detail = fft3d_plan_last_error(plan) if plan else ""
        raise FFT3DError(rc, where, detail)


# ------------------------------------------------------------ raw C ABI
def fft3d_plan_create(n0, n1, n2, dtype):
    h = ctypes.c_void_p()
    _check(load_library().fft3d_plan_create(ctypes.byref(h), n0, n1, n2, dtype), "fft3d_plan_create")
    return h.value


def fft3d_plan_create_batched(batch, n0, n1, n2, dtype):
    h = ctypes.c_void_p()
    _check(load_library().fft3d_plan_create_batched(ctypes.byref(h), batch, n0, n1, n2, dtype),
           "fft3d_plan_create_batched")
    return h.value


def fft3d_plan_destroy(plan):
    _check(load_library().fft3d_plan_destroy(plan), "fft3d_plan_destroy")


def fft3d_exec_r2c(plan, in_real, out_cplx, stream):
    _check(load_library().fft3d_exec_r2c(plan, in_real, out_cplx, stream), "fft3d_exec_r2c", plan)


def fft3d_exec_c2r(plan, in_cplx, out_real, stream):
    _check(load_library().fft3d_exec_c2r(plan, in_cplx, out_real, stream), "fft3d_exec_c2r", plan)


def fft3d_exec_c2r_overwrite(plan, inout_cplx, out_real, stream):
    _check(load_library().fft3d_exec_c2r_overwrite(plan, inout_cplx, out_real, stream),
           "fft3d_exec_c2r_overwrite", plan)


def fft3d_exec_r2c_adjoint(plan, in_cplx, out_real, stream):
    _check(load_library().fft3d_exec_r2c_adjoint(plan, in_cplx, out_real, stream),
           "fft3d_exec_r2c_adjoint", plan)


def fft3d_exec_c2r_adjoint(plan, in_real, out_cplx, stream):
    _check(load_library().fft3d_exec_c2r_adjoint(plan, in_real, out_cplx, stream),
           "fft3d_exec_c2r_adjoint", plan)


def fft3d_strerror(status):
    return load_library().fft3d_strerror(int(status)).decode()


def fft3d_plan_last_error(plan):
    return load_library().fft3d_plan_last_error(plan).decode()


def fft3d_supported_length(n, axis):
    return bool(load_library().fft3d_supported_length(n, axis))


def fft3d_plan_set_profiling(plan, enable):
    _check(load_library().fft3d_plan_set_profiling(plan, 1 if enable else 0), "fft3d_plan_set_profiling")


def fft3d_plan_profile_read(plan, max_entries=16):
    arr = (KernelStat * max_entries)()
    cnt = ctypes.c_int()
    _check(load_library().fft3d_plan_profile_read(plan, arr, max_entries, ctypes.byref(cnt)),
           "fft3d_plan_profile_read", plan)
    return [{"name": arr[i].name.decode(), "launches": arr[i].launches, "total_ms": arr[i].total_ms,
             "bytes_per_launch": arr[i].bytes_per_launch} for i in range(cnt.value)]


def fft3d_plan_launch_count(plan):
    c = ctypes.c_int64()
    _check(load_library().fft3d_plan_launch_count(plan, ctypes.byref(c)), "fft3d_plan_launch_count")
    return c.value


def fft3d_plan_status(plan):
    """Device error flag (0/1) of the plan's bounded waits; synchronises and clears it."""
    v = ctypes.c_int()
    _check(load_library().fft3d_plan_status(plan, ctypes.byref(v)), "fft3d_plan_status", plan)
    return v.value


def fft3d_plan_set_debug(plan, inject_stall, spin_limit=0):
    _check(load_library().fft3d_plan_set_debug(plan, 1 if inject_stall else 0, int(spin_limit)),
           "fft3d_plan_set_debug")


def fft3d_plan_info(plan):
    v = ctypes.c_int()
    _check(load_library().fft3d_plan_info(plan, ctypes.byref(v)), "fft3d_plan_info")
    return {"fused_plane_pass": bool(v.value)}


def fft3d_plan_set_fused(plan, enable):
    _check(load_library().fft3d_plan_set_fused(plan, 1 if enable else 0), "fft3d_plan_set_fused", plan)


def fft3d_exec_c2r_noalloc(in_cplx, out_real, n0, n1, n2, dtype, stream):
    """Plan-free inverse C2R that allocates nothing (for callers that cannot
    call cudaMalloc); see include/fft3d.h for the shared-scratch rules."""
    _check(load_library().fft3d_exec_c2r_noalloc(in_cplx, out_real, n0, n1, n2, dtype, stream),
           "fft3d_exec_c2r_noalloc")


def fft3d_noalloc_status():
    """Device error word (0/1) of fft3d_exec_c2r_noalloc on the current
    device; synchronises the device and clears it."""
    v = ctypes.c_int()
    _check(load_library().fft3d_noalloc_status(ctypes.byref(v)), "fft3d_noalloc_status")
    return v.value


def fft3d_measure_fp64_peak():
    """Measured FP64 GFLOP/s of the current device for FMA (2 flops each),
    add and multiply chains (see include/fft3d.h)."""
    f, a, m = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load_library().fft3d_measure_fp64_peak(ctypes.byref(f), ctypes.byref(a), ctypes.byref(m)),
           "fft3d_measure_fp64_peak")
    return {"fma_gflops": f.value, "add_gflops": a.value, "mul_gflops": m.value}


# ------------------------------------------------------------ torch layer
def _torch():
    import torch
    return torch


def _dtype_code(real_dtype):
    torch = _torch()
    if real_dtype == torch.float32:
        return FFT3D_F32
    if real_dtype == torch.float64:
        return FFT3D_F64
    raise FFT3DError(FFT3D_ERR_DTYPE, "dtype", str(real_dtype))


def complex_of(real_dtype):
    torch = _torch()
    return torch.complex64 if real_dtype == torch.float32 else torch.complex128


def real_of(complex_dtype):
    torch = _torch()
    return torch.float32 if complex_dtype == torch.complex64 else torch.float64


class Plan:
    """An fft3d plan for one (N0, N1, N2, dtype) on one CUDA device.  With
    batch > 1 every call transforms `batch` fields: tensors carry a leading
    batch dimension ([B, N0, N1, N2] real, [B, N0, N1, N2/2+1] complex)."""

    def __init__(self, shape, dtype, device=None, batch=1):
        torch = _torch()
        self.shape = tuple(int(s) for s in shape)
        self.batch = int(batch)
        self.lead = (self.batch,) if self.batch > 1 else ()
        self.real_dtype = dtype
        self.complex_dtype = complex_of(dtype)
        self.device = torch.device(device if device is not None else "cuda", )
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(self.device):
            self.handle = fft3d_plan_create_batched(self.batch, *self.shape, _dtype_code(dtype))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                fft3d_plan_destroy(h)
            except Exception:
                pass
            self.handle = None

    @property
    def half_shape(self):
        n0, n1, n2 = self.shape
        return self.lead + (n0, n1, n2 // 2 + 1)

    @property
    def real_shape(self):
        return self.lead + self.shape

    def _stream(self):
        return _torch().cuda.current_stream(self.device).cuda_stream

    def _run(self, fn, src, dst):
        torch = _torch()
        with torch.cuda.device(self.device):
            fn(self.handle, src.data_ptr(), dst.data_ptr(), self._stream())

    def empty_real(self):
        return _torch().empty(self.real_shape, dtype=self.real_dtype, device=self.device)

    def empty_complex(self):
        return _torch().empty(self.half_shape, dtype=self.complex_dtype, device=self.device)

    def empty_padded(self):
        """Real buffer with rows padded to 2 (N2/2 + 1): the in-place layout."""
        n0, n1, n2 = self.shape
        return _torch().empty(self.lead + (n0, n1, 2 * (n2 // 2 + 1)), dtype=self.real_dtype,
                              device=self.device)

    def _check_real(self, t, padded=False, host_ok=False):
        n0, n1, n2 = self.shape
        want = self.lead + ((n0, n1, 2 * (n2 // 2 + 1)) if padded else self.shape)
        where_ok = t.device == self.device or (host_ok and t.device.type == "cpu" and t.is_pinned())
        if t.dtype != self.real_dtype or tuple(t.shape) != want or not t.is_contiguous() or not where_ok:
            raise FFT3DError(FFT3D_ERR_ARG, "real tensor", f"need contiguous {want} {self.real_dtype} on {self.device}")

    def _check_cplx(self, t):
        if (t.dtype != self.complex_dtype or tuple(t.shape) != self.half_shape or not t.is_contiguous()
                or t.device != self.device):
            raise FFT3DError(FFT3D_ERR_ARG, "complex tensor",
                             f"need contiguous {self.half_shape} {self.complex_dtype} on {self.device}")

    # out-of-place; x may also be a pinned host tensor (read once, by the first pass)
    def r2c(self, x, out=None):
        self._check_real(x, host_ok=True)
        out = self.empty_complex() if out is None else out
        self._check_cplx(out)
        self._run(fft3d_exec_r2c, x, out)
        return out

    def c2r(self, X, out=None):
        self._check_cplx(X)
        out = self.empty_real() if out is None else out
        self._check_real(out)
        self._run(fft3d_exec_c2r, X, out)
        return out

    def c2r_overwrite(self, X, out=None):
        """Inverse that uses X as work space (X is overwritten); `out` may be a
        pinned host tensor (written once, by the last pass)."""
        self._check_cplx(X)
        out = self.empty_real() if out is None else out
        self._check_real(out, host_ok=True)
        self._run(fft3d_exec_c2r_overwrite, X, out)
        return out

    def r2c_adjoint(self, G, out=None):
        self._check_cplx(G)
        out = self.empty_real() if out is None else out
        self._check_real(out)
        self._run(fft3d_exec_r2c_adjoint, G, out)
        return out

    def c2r_adjoint(self, g, out=None):
        self._check_real(g)
        out = self.empty_complex() if out is None else out
        self._check_cplx(out)
        self._run(fft3d_exec_c2r_adjoint, g, out)
        return out

    # in place on a padded real buffer; returns the complex / real view
    def r2c_(self, buf):
        self._check_real(buf, padded=True)
        self._run(fft3d_exec_r2c, buf, buf)
        return buf.view(self.complex_dtype)

    def c2r_(self, buf):
        """buf: the padded real buffer (or its complex view) holding a half spectrum."""
        if buf.is_complex():
            buf = buf.view(self.real_dtype)
        self._check_real(buf, padded=True)
        self._run(fft3d_exec_c2r, buf, buf)
        return buf

    def set_profiling(self, enable):
        fft3d_plan_set_profiling(self.handle, enable)

    def profile_read(self):
        with _torch().cuda.device(self.device):
            return fft3d_plan_profile_read(self.handle)

    def launch_count(self):
        return fft3d_plan_launch_count(self.handle)

    def status(self):
        with _torch().cuda.device(self.device):
            return fft3d_plan_status(self.handle)

    def set_debug(self, inject_stall, spin_limit=0):
        fft3d_plan_set_debug(self.handle, inject_stall, spin_limit)

    def info(self):
        return fft3d_plan_info(self.handle)

    def set_fused(self, enable):
        fft3d_plan_set_fused(self.handle, enable)


_plans = {}
_plans_lock = threading.Lock()


def get_plan(shape, dtype, device, batch=1):
    """The cached plan for (shape, dtype, device, batch) on the device's
    current torch stream.  A plan serves one stream at a time (its scratch
    plane and tile counter are shared by its calls), so each stream gets a
    plan of its own."""
    torch = _torch()
    device = torch.device(device)
    if device.index is None:
        device = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(device).cuda_stream
    key = (tuple(int(s) for s in shape), dtype, device.index, int(batch), stream)
    with _plans_lock:
        p = _plans.get(key)
        if p is None:
            p = Plan(shape, dtype, device, batch)
            _plans[key] = p
    return p


def _split_batch(shape):
    """(batch, field shape) of a 3D shape or a 4D [B, N0, N1, N2] shape."""
    shape = tuple(int(s) for s in shape)
    if len(shape) == 4:
        return shape[0], shape[1:]
    if len(shape) == 3:
        return 1, shape
    raise FFT3DError(FFT3D_ERR_ARG, "shape", f"need (N0, N1, N2) or (B, N0, N1, N2), got {shape}")


def _make_autograd():
    torch = _torch()

    # each pass looks its plan up on the stream it runs on (the backward may run on another)
    class RFFT3(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x):
            b, shape = _split_batch(x.shape)
            ctx.key = (shape, x.dtype, x.device, b)
            return get_plan(*ctx.key).r2c(x.contiguous())

        @staticmethod
        def backward(ctx, G):
            return get_plan(*ctx.key).r2c_adjoint(G.contiguous())

    class IRFFT3(torch.autograd.Function):
        @staticmethod
        def forward(ctx, X, shape):
            b, shape = _split_batch(shape)
            ctx.key = (shape, real_of(X.dtype), X.device, b)
            return get_plan(*ctx.key).c2r(X.contiguous())

        @staticmethod
        def backward(ctx, g):
            return get_plan(*ctx.key).c2r_adjoint(g.contiguous()), None

    return RFFT3, IRFFT3


_autograd = None


def rfft3(x):
    """Forward R2C (Eq. 1) of a real [N0][N1][N2] CUDA tensor, or of each field
    of a [B][N0][N1][N2] batch; differentiable."""
    global _autograd
    if _autograd is None:
        _autograd = _make_autograd()
    return _autograd[0].apply(x)


def irfft3(X, shape):
    """Normalised inverse C2R (Eq. 2 and 1/N^3) to real `shape` ((N0, N1, N2),
    or (B, N0, N1, N2) for a batch of fields); differentiable."""
    global _autograd
    if _autograd is None:
        _autograd = _make_autograd()
    return _autograd[1].apply(X, tuple(int(s) for s in shape))

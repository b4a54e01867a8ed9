"""ctypes binding of liblinmin.so (C ABI in include/linmin.h).

Argument marshalling only: every function forwards to the C entry point of
the same name; all arithmetic runs in the library's CUDA kernels.  Arrays
may be torch tensors (CUDA or CPU) or numpy arrays (host); they must be
contiguous float32 (int32 for ``iterations``).  There is no CPU fallback:
importing this module fails when the library cannot be loaded.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

LINMIN_OK = 0
LINMIN_ERR_INVALID = 1
LINMIN_ERR_OOM = 2
LINMIN_ERR_CUDA = 3
LINMIN_ERR_RANK = 4
LINMIN_ERR_TIMEOUT = 5
LINMIN_ERR_NOT_CONVERGED = 6
LINMIN_ERR_UNSUPPORTED = 7
LINMIN_PROJ_DF = 0
LINMIN_STO = 0
LINMIN_SLO = 1
LINMIN_POS = 2
LINMIN_POS_SCALE = 64
LINMIN_MAX_P = 64
LINMIN_MAX_L = 4096

STATUS_NAMES = {0: "OK", 1: "ERR_INVALID", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_RANK",
                5: "ERR_TIMEOUT", 6: "ERR_NOT_CONVERGED", 7: "ERR_UNSUPPORTED"}

EXPORTED = ("linmin_default_options", "linmin_create", "linmin_unmix", "linmin_wait",
            "linmin_phase_times", "linmin_destroy", "linmin_last_error", "linmin_version",
            "linmin_unmix_noalloc", "linmin_last_launches", "linmin_phase_times_at",
            "linmin_server_default_options", "linmin_server_create", "linmin_server_submit",
            "linmin_server_poll", "linmin_server_wait", "linmin_server_get_stats",
            "linmin_server_last_error", "linmin_server_destroy", "linmin_server_handle_bytes",
            "linmin_get_lanes", "linmin_set_lanes", "linmin_autotune", "linmin_unmix_cov",
            "linmin_extra_spectra", "linmin_detect", "linmin_threshold_stats",
            "linmin_thresholds", "linmin_autofit", "linmin_second_pass",
            "linmin_unmix_masked", "linmin_noalloc_scratch_bytes", "linmin_fp32_peak",
            "linmin_live_allocations", "linmin_unmix_batch")
LINMIN_NOALLOC_SCRATCH_MB = 64
LINMIN_PHASE_RING = 32
LINMIN_PROJ_TC = 1
LINMIN_PROJ_BF16 = 2
PHASES = ("prep", "project", "ipm", "crossover", "retry", "rms")


class linmin_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("constraint", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("tol", ctypes.c_float),
                ("refine_mu", ctypes.c_float), ("cuda_stream", ctypes.c_void_p),
                ("profile", ctypes.c_int)]


class linmin_server_options(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_ulonglong), ("slots", ctypes.c_int),
                ("chunk_pixels", ctypes.c_longlong), ("max_iter", ctypes.c_int),
                ("autotune", ctypes.c_int)]


class linmin_request(ctypes.Structure):
    _fields_ = [("library", ctypes.c_void_p), ("L", ctypes.c_int), ("P", ctypes.c_int),
                ("cube", ctypes.c_void_p), ("N", ctypes.c_longlong), ("sigma", ctypes.c_void_p),
                ("abundances", ctypes.c_void_p), ("uncertainties", ctypes.c_void_p),
                ("residual_rms", ctypes.c_void_p), ("iterations", ctypes.c_void_p)]


class linmin_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_ulonglong) for n in
                ("requests", "requests_done", "chunks", "handles_created", "evictions",
                 "bytes", "peak_bytes")] + [("running", ctypes.c_int),
                                            ("max_running", ctypes.c_int),
                                            ("libraries", ctypes.c_longlong),
                                            ("autotuned", ctypes.c_longlong)]


_I64x = ctypes.c_longlong * LINMIN_MAX_P
_F64x = ctypes.c_double * LINMIN_MAX_P


class linmin_detection(ctypes.Structure):
    _fields_ = [("count", _I64x), ("argmax", _I64x), ("n_true", _I64x), ("true_pos", _I64x),
                ("false_pos", _I64x), ("xsum", _F64x), ("xmax", ctypes.c_float * LINMIN_MAX_P),
                ("key", ctypes.c_ulonglong * LINMIN_MAX_P)]


class linmin_threshold_sums(ctypes.Structure):
    _fields_ = [("n_pos", _I64x), ("n_neg", _I64x), ("sum_pos", _F64x), ("m2_pos", _F64x),
                ("sum_neg", _F64x), ("m2_neg", _F64x)]


class LinminError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None, build_if_missing: bool = True) -> ctypes.CDLL:
    """Load liblinmin.so (building it in-tree first if it is missing)."""
    if path is None and build_if_missing:
        path = _build.build()             # no-op when the stamp matches the sources
    path = path or _build.LIB
    if not os.path.exists(path):
        raise OSError(f"{path} not built")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    P = ctypes.c_void_p
    lib.linmin_default_options.argtypes = [ctypes.POINTER(linmin_options)]
    lib.linmin_default_options.restype = ctypes.c_int
    lib.linmin_create.argtypes = [P, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(linmin_options), ctypes.POINTER(H)]
    lib.linmin_create.restype = ctypes.c_int
    lib.linmin_unmix.argtypes = [H, P, ctypes.c_longlong, P, P, P, P, P]
    lib.linmin_unmix.restype = ctypes.c_int
    lib.linmin_unmix_cov.argtypes = [H, P, ctypes.c_longlong, P, P, P, P, P]
    lib.linmin_unmix_cov.restype = ctypes.c_int
    PP_ = ctypes.POINTER(ctypes.c_void_p)
    lib.linmin_unmix_batch.argtypes = [ctypes.c_int, PP_, PP_, ctypes.POINTER(ctypes.c_longlong), PP_,
                                       PP_, PP_, PP_, PP_]
    lib.linmin_unmix_batch.restype = ctypes.c_int
    lib.linmin_wait.argtypes = [H, ctypes.POINTER(ctypes.c_longlong)]
    lib.linmin_wait.restype = ctypes.c_int
    lib.linmin_phase_times.argtypes = [H, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
    lib.linmin_phase_times.restype = ctypes.c_int
    lib.linmin_destroy.argtypes = [H]
    lib.linmin_destroy.restype = ctypes.c_int
    lib.linmin_last_error.argtypes = [H]
    lib.linmin_last_error.restype = ctypes.c_char_p
    lib.linmin_unmix_noalloc.argtypes = [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_longlong,
                                         P, P, P, P, P, ctypes.c_void_p]
    lib.linmin_unmix_noalloc.restype = ctypes.c_int
    lib.linmin_noalloc_scratch_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                                 ctypes.POINTER(ctypes.c_ulonglong)]
    lib.linmin_noalloc_scratch_bytes.restype = ctypes.c_int
    lib.linmin_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    lib.linmin_fp32_peak.restype = ctypes.c_int
    lib.linmin_live_allocations.argtypes = [ctypes.POINTER(ctypes.c_longlong)]
    lib.linmin_live_allocations.restype = ctypes.c_int
    SV = ctypes.c_void_p
    lib.linmin_server_default_options.argtypes = [ctypes.POINTER(linmin_server_options)]
    lib.linmin_server_default_options.restype = ctypes.c_int
    lib.linmin_server_create.argtypes = [ctypes.POINTER(linmin_server_options),
                                         ctypes.POINTER(SV)]
    lib.linmin_server_create.restype = ctypes.c_int
    lib.linmin_server_submit.argtypes = [SV, ctypes.POINTER(linmin_request),
                                         ctypes.POINTER(ctypes.c_longlong)]
    lib.linmin_server_submit.restype = ctypes.c_int
    lib.linmin_server_poll.argtypes = [SV, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]
    lib.linmin_server_poll.restype = ctypes.c_int
    lib.linmin_server_wait.argtypes = [SV, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double)]
    lib.linmin_server_wait.restype = ctypes.c_int
    lib.linmin_server_get_stats.argtypes = [SV, ctypes.POINTER(linmin_server_stats)]
    lib.linmin_server_get_stats.restype = ctypes.c_int
    lib.linmin_server_last_error.argtypes = [SV]
    lib.linmin_server_last_error.restype = ctypes.c_char_p
    lib.linmin_server_handle_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                               ctypes.c_int]
    lib.linmin_server_handle_bytes.restype = ctypes.c_ulonglong
    lib.linmin_server_destroy.argtypes = [SV]
    lib.linmin_server_destroy.restype = ctypes.c_int
    lib.linmin_phase_times_at.argtypes = [H, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                          ctypes.c_int]
    lib.linmin_phase_times_at.restype = ctypes.c_int
    lib.linmin_get_lanes.argtypes = [H]
    lib.linmin_get_lanes.restype = ctypes.c_int
    lib.linmin_set_lanes.argtypes = [H, ctypes.c_int]
    lib.linmin_set_lanes.restype = ctypes.c_int
    lib.linmin_autotune.argtypes = [H, P, ctypes.c_longlong, P, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int)]
    lib.linmin_autotune.restype = ctypes.c_int
    lib.linmin_last_launches.argtypes = [H]
    lib.linmin_last_launches.restype = ctypes.c_int
    lib.linmin_version.argtypes = []
    lib.linmin_version.restype = ctypes.c_char_p
    lib.linmin_extra_spectra.argtypes = [ctypes.c_int, P, ctypes.c_int, P]
    lib.linmin_extra_spectra.restype = ctypes.c_int
    lib.linmin_detect.argtypes = [P, P, P, P, P, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                  P, ctypes.c_float, P, P, ctypes.c_void_p]
    lib.linmin_detect.restype = ctypes.c_int
    lib.linmin_threshold_stats.argtypes = [P, P, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                           P, ctypes.c_void_p]
    lib.linmin_threshold_stats.restype = ctypes.c_int
    lib.linmin_thresholds.argtypes = [ctypes.POINTER(linmin_threshold_sums), ctypes.c_int, P]
    lib.linmin_thresholds.restype = ctypes.c_int
    lib.linmin_autofit.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P,
                                   ctypes.c_void_p]
    lib.linmin_autofit.restype = ctypes.c_int
    lib.linmin_second_pass.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(linmin_options), P, ctypes.c_longlong, P,
                                       P, P, P, P, P]
    lib.linmin_second_pass.restype = ctypes.c_int
    lib.linmin_unmix_masked.argtypes = [H, P, ctypes.c_longlong, P, P, ctypes.c_int, P, P, P, P]
    lib.linmin_unmix_masked.restype = ctypes.c_int
    return lib


_LIB = None


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def _ptr(a, dtype_name: str = "float32"):
    """Raw pointer of a contiguous torch tensor / numpy array (or None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):          # torch.Tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if str(a.dtype).split(".")[-1] != dtype_name:
            raise TypeError(f"expected {dtype_name}, got {a.dtype}")
        return ctypes.c_void_p(a.data_ptr())
    if hasattr(a, "ctypes"):            # numpy.ndarray
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if a.dtype.name != dtype_name:
            raise TypeError(f"expected {dtype_name}, got {a.dtype}")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _check(status: int, handle=None):
    if status != LINMIN_OK:
        raise LinminError(status, linmin_last_error(handle))
    return status


def linmin_default_options() -> linmin_options:
    o = linmin_options()
    _check(lib().linmin_default_options(ctypes.byref(o)))
    return o


def linmin_create(library, L: int, P: int, opt: linmin_options | None = None) -> ctypes.c_void_p:
    """Handle for a P x L float32 library (host or device)."""
    h = ctypes.c_void_p()
    st = lib().linmin_create(_ptr(library), int(L), int(P),
                             ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    _check(st, None)
    return h


def linmin_unmix(h, cube, N: int, sigma, abundances=None, uncertainties=None,
                 residual_rms=None, iterations=None, check: bool = True) -> int:
    st = lib().linmin_unmix(h, _ptr(cube), int(N), _ptr(sigma), _ptr(abundances),
                            _ptr(uncertainties), _ptr(residual_rms),
                            _ptr(iterations, "int32"))
    if check and st not in (LINMIN_OK, LINMIN_ERR_NOT_CONVERGED):
        _check(st, h)
    return st


def linmin_unmix_batch(handles, cubes, Ns, sigmas, abundances, uncertainties=None,
                       residual_rms=None, iterations=None, check: bool = True) -> int:
    """linmin_unmix of several cubes with one interior-point launch per
    group of equal P (device tensors; lists of equal length, entries of the
    optional lists may be None)."""
    n = len(handles)
    arr = lambda vals: (ctypes.c_void_p * n)(*vals)
    opt = lambda lst, dt="float32": None if lst is None else arr([_ptr(a, dt) for a in lst])
    st = lib().linmin_unmix_batch(n, arr(handles), arr([_ptr(c) for c in cubes]),
                                  (ctypes.c_longlong * n)(*[int(v) for v in Ns]),
                                  arr([_ptr(sg) for sg in sigmas]), arr([_ptr(x) for x in abundances]),
                                  opt(uncertainties), opt(residual_rms), opt(iterations, "int32"))
    if check and st not in (LINMIN_OK, LINMIN_ERR_NOT_CONVERGED):
        _check(st, handles[0])
    return st


def linmin_unmix_cov(h, cube, N: int, cov_inv, abundances=None, uncertainties=None,
                     residual_rms=None, iterations=None, check: bool = True) -> int:
    """linmin_unmix under a full noise covariance (cov_inv: L x L float64)."""
    st = lib().linmin_unmix_cov(h, _ptr(cube), int(N), _ptr(cov_inv, "float64"),
                                _ptr(abundances), _ptr(uncertainties), _ptr(residual_rms),
                                _ptr(iterations, "int32"))
    if check and st not in (LINMIN_OK, LINMIN_ERR_NOT_CONVERGED):
        _check(st, h)
    return st


def linmin_wait(h) -> tuple[int, int]:
    n = ctypes.c_longlong(0)
    st = lib().linmin_wait(h, ctypes.byref(n))
    return st, int(n.value)


def linmin_phase_times(h) -> dict:
    """Per-phase device milliseconds of the last linmin_unmix (profile mode)."""
    arr = (ctypes.c_float * len(PHASES))()
    _check(lib().linmin_phase_times(h, arr, len(PHASES)), h)
    return {k: float(v) for k, v in zip(PHASES, arr)}


def linmin_phase_times_at(h, back: int) -> dict:
    """Per-phase device milliseconds of the call `back` calls before the last."""
    arr = (ctypes.c_float * len(PHASES))()
    _check(lib().linmin_phase_times_at(h, back, arr, len(PHASES)), h)
    return {k: float(v) for k, v in zip(PHASES, arr)}


def linmin_destroy(h) -> int:
    return lib().linmin_destroy(h)


def linmin_last_error(h=None) -> str:
    s = lib().linmin_last_error(h)
    return s.decode() if s else ""


def linmin_unmix_noalloc(library, L: int, P: int, cube, N: int, sigma, abundances=None,
                         uncertainties=None, residual_rms=None, iterations=None,
                         stream=None) -> int:
    """The allocation-free variant (device pointers only); returns the status."""
    st = None if stream is None else ctypes.c_void_p(int(stream))
    return lib().linmin_unmix_noalloc(_ptr(library), int(L), int(P), _ptr(cube), int(N),
                                      _ptr(sigma), _ptr(abundances), _ptr(uncertainties),
                                      _ptr(residual_rms), _ptr(iterations, "int32"), st)


def linmin_noalloc_scratch_bytes(L: int, P: int, N: int) -> tuple[int, int]:
    """(status, bytes) of linmin_unmix_noalloc's scratch for (L, P, N)."""
    b = ctypes.c_ulonglong(0)
    st = lib().linmin_noalloc_scratch_bytes(int(L), int(P), int(N), ctypes.byref(b))
    return st, int(b.value)


def linmin_live_allocations() -> int:
    """Device allocations the library's handles hold now."""
    n = ctypes.c_longlong(0)
    _check(lib().linmin_live_allocations(ctypes.byref(n)))
    return n.value


def linmin_fp32_peak(stream=None) -> tuple[float, float]:
    """Measured (FFMA, FFMA2) TFLOP/s of the current device."""
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().linmin_fp32_peak(ctypes.byref(a), ctypes.byref(b), _stream_ptr(stream)))
    return a.value, b.value


def linmin_get_lanes(h) -> int:
    """Lanes per pixel of the handle's interior-point kernel."""
    return lib().linmin_get_lanes(h)


def linmin_set_lanes(h, lanes: int) -> int:
    return _check(lib().linmin_set_lanes(h, int(lanes)), h)


def linmin_autotune(h, cube, N: int, sigma) -> tuple[int, list]:
    """Time every compiled bucket for the handle's P on a sample of the cube
    and keep the fastest; returns (lanes per pixel, per-candidate ms)."""
    lanes = ctypes.c_int(0)
    n = ctypes.c_int(0)
    ms = (ctypes.c_float * 16)()
    _check(lib().linmin_autotune(h, _ptr(cube), int(N), _ptr(sigma), ctypes.byref(lanes), ms, 16,
                                 ctypes.byref(n)), h)
    return lanes.value, [float(ms[i]) for i in range(n.value)]


def linmin_last_launches(h) -> int:
    """Kernel launches queued by the last linmin_unmix on h."""
    return lib().linmin_last_launches(h)


def linmin_version() -> str:
    return lib().linmin_version().decode()


def _ptr_any(a, names):
    """_ptr accepting any of the dtype names (bit masks: int64 or uint64)."""
    if a is None:
        return None
    got = str(a.dtype).split(".")[-1] if hasattr(a, "data_ptr") else a.dtype.name
    if got not in names:
        raise TypeError(f"expected one of {names}, got {got}")
    return _ptr(a, got)


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


def linmin_extra_spectra(L: int, n_extras: int = 12, wavelengths=None):
    """The paper's additional spectra, (n_extras, L) float32 numpy."""
    import numpy as np
    out = np.empty((n_extras, L), dtype=np.float32)
    w = None if wavelengths is None else np.ascontiguousarray(wavelengths, dtype=np.float32)
    _check(lib().linmin_extra_spectra(int(L), _ptr(w), int(n_extras), _ptr(out)))
    return out


def linmin_detect(x, sx, rms, iterations, truth, N: int, P: int, n_minerals: int, x_min,
                  rms_max: float, mask=None, out=None, stream=None) -> int:
    """Queue the detection kernel (device arrays; out: a device byte buffer
    of sizeof(linmin_detection), see detection_summary)."""
    import numpy as np
    xm = np.ascontiguousarray(np.asarray(x_min, dtype=np.float32).reshape(-1))
    return _check(lib().linmin_detect(_ptr(x), _ptr(sx), _ptr(rms), _ptr(iterations, "int32"),
                                      _ptr_any(truth, ("int64", "uint64")), int(N), int(P),
                                      int(n_minerals), _ptr(xm), float(rms_max),
                                      _ptr_any(mask, ("int64", "uint64")),
                                      _ptr(out, "uint8"), _stream_ptr(stream)))


def linmin_threshold_stats(x, truth, N: int, P: int, n_minerals: int, out, stream=None) -> int:
    """Queue the threshold sums (out: a device byte buffer of
    sizeof(linmin_threshold_sums))."""
    return _check(lib().linmin_threshold_stats(_ptr(x), _ptr_any(truth, ("int64", "uint64")),
                                               int(N), int(P), int(n_minerals),
                                               _ptr(out, "uint8"), _stream_ptr(stream)))


def linmin_thresholds(sums: linmin_threshold_sums, n_minerals: int):
    """eq. Threshold from sums on the host; float32 numpy of n_minerals."""
    import numpy as np
    c = np.empty(max(1, n_minerals), dtype=np.float32)
    _check(lib().linmin_thresholds(ctypes.byref(sums), int(n_minerals), _ptr(c)))
    return c[:n_minerals]


def linmin_autofit(library, L: int, P: int, resid_ls=None, resid_nn=None, coef_nn=None,
                   rms_ls=None, rms_nn=None, status=None, stream=None) -> int:
    """Queue the library auto-fit (device arrays)."""
    return _check(lib().linmin_autofit(_ptr(library), int(L), int(P), _ptr(resid_ls),
                                       _ptr(resid_nn), _ptr(coef_nn), _ptr(rms_ls),
                                       _ptr(rms_nn), _ptr(status, "int32"),
                                       _stream_ptr(stream)))


def linmin_second_pass(library, L: int, P: int, n_minerals: int, cube, N: int, sigma, mask,
                       abundances=None, uncertainties=None, residual_rms=None, iterations=None,
                       opt: linmin_options | None = None) -> int:
    """Second pass with the detected spectra (device arrays; synchronous).
    Returns LINMIN_OK or LINMIN_ERR_NOT_CONVERGED; other errors raise."""
    st = lib().linmin_second_pass(_ptr(library), int(L), int(P), int(n_minerals),
                                  ctypes.byref(opt) if opt is not None else None, _ptr(cube),
                                  int(N), _ptr(sigma), _ptr_any(mask, ("int64", "uint64")),
                                  _ptr(abundances), _ptr(uncertainties), _ptr(residual_rms),
                                  _ptr(iterations, "int32"))
    if st not in (LINMIN_OK, LINMIN_ERR_NOT_CONVERGED):
        _check(st)
    return st


def linmin_unmix_masked(h, cube, N: int, sigma, mask, n_minerals: int, abundances=None,
                        uncertainties=None, residual_rms=None, iterations=None) -> int:
    """Unmix with per-pixel library subsets (mask: device bit masks)."""
    return _check(lib().linmin_unmix_masked(h, _ptr(cube), int(N), _ptr(sigma),
                                            _ptr_any(mask, ("int64", "uint64")),
                                            int(n_minerals), _ptr(abundances),
                                            _ptr(uncertainties), _ptr(residual_rms),
                                            _ptr(iterations, "int32")), h)


def _struct_from(buf, cls):
    data = buf.cpu().numpy().tobytes() if hasattr(buf, "cpu") else bytes(buf)
    return cls.from_buffer_copy(data)


def detection_summary(buf) -> dict:
    """Decode a linmin_detection byte buffer (device or host) into numpy arrays."""
    import numpy as np
    d = _struct_from(buf, linmin_detection)
    out = {f: np.array(getattr(d, f)) for f, _ in linmin_detection._fields_ if f != "key"}
    return out


def threshold_sums(buf) -> linmin_threshold_sums:
    """Decode a linmin_threshold_sums byte buffer (device or host)."""
    return _struct_from(buf, linmin_threshold_sums)


class Unmixer:
    """Convenience owner of a handle; outputs are allocated as torch tensors
    on the device of the inputs (plumbing only)."""

    def __init__(self, library, max_iter: int = 100, tol: float = 1e-9,
                 refine_mu: float = 1e-9, stream=None, profile: bool = False,
                 precision: int | None = None, constraint: int = 0):
        import torch
        S = library if hasattr(library, "data_ptr") else torch.as_tensor(library)
        S = S.to(torch.float32).contiguous()
        self.P, self.L = int(S.shape[0]), int(S.shape[1])
        opt = linmin_default_options()
        opt.max_iter, opt.tol, opt.refine_mu = int(max_iter), float(tol), float(refine_mu)
        opt.profile = int(bool(profile))
        if precision is not None:
            opt.precision = int(precision)
        opt.constraint = int(constraint)
        if stream is not None:
            opt.cuda_stream = ctypes.c_void_p(int(stream.cuda_stream))
        self.h = linmin_create(S, self.L, self.P, opt)

    def __call__(self, cube, sigma):
        import torch
        N = int(cube.shape[0])
        dev = cube.device
        x = torch.empty((N, self.P), dtype=torch.float32, device=dev)
        sx = torch.empty((N, self.P), dtype=torch.float32, device=dev)
        rms = torch.empty((N,), dtype=torch.float32, device=dev)
        it = torch.empty((N,), dtype=torch.int32, device=dev)
        linmin_unmix(self.h, cube, N, sigma, x, sx, rms, it)
        return x, sx, rms, it

    def wait(self):
        return linmin_wait(self.h)

    def phase_times(self):
        return linmin_phase_times(self.h)

    def close(self):
        if self.h:
            linmin_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving
def linmin_server_default_options() -> linmin_server_options:
    o = linmin_server_options()
    _check(lib().linmin_server_default_options(ctypes.byref(o)))
    return o


def linmin_server_create(opt: linmin_server_options | None = None):
    s = ctypes.c_void_p()
    st = lib().linmin_server_create(ctypes.byref(opt) if opt is not None else None,
                                    ctypes.byref(s))
    if st != LINMIN_OK:
        raise LinminError(st, "linmin_server_create failed")
    return s


def linmin_server_submit(s, library, L: int, P: int, cube, N: int, sigma, abundances=None,
                         uncertainties=None, residual_rms=None, iterations=None) -> int:
    """Queue one cube; returns its ticket (raises on a rejected request)."""
    r = linmin_request(_ptr(library), int(L), int(P), _ptr(cube), int(N), _ptr(sigma),
                       _ptr(abundances), _ptr(uncertainties), _ptr(residual_rms),
                       _ptr(iterations, "int32"))
    t = ctypes.c_longlong(0)
    st = lib().linmin_server_submit(s, ctypes.byref(r), ctypes.byref(t))
    if st != LINMIN_OK:
        raise LinminError(st, linmin_server_last_error(s))
    return t.value


def linmin_server_poll(s, ticket: int) -> bool:
    d = ctypes.c_int(0)
    _check(lib().linmin_server_poll(s, int(ticket), ctypes.byref(d)))
    return bool(d.value)


def linmin_server_wait(s, ticket: int) -> tuple[int, float]:
    """(status, latency in ms from submit to completion) of a request."""
    ms = ctypes.c_double(0.0)
    st = lib().linmin_server_wait(s, int(ticket), ctypes.byref(ms))
    return st, ms.value


def linmin_server_get_stats(s) -> dict:
    st = linmin_server_stats()
    _check(lib().linmin_server_get_stats(s, ctypes.byref(st)))
    return {n: getattr(st, n) for n, _ in linmin_server_stats._fields_}


def linmin_server_last_error(s) -> str:
    m = lib().linmin_server_last_error(s)
    return m.decode() if m else ""


def linmin_server_handle_bytes(L: int, P: int, chunk_pixels: int, host_io: bool = False) -> int:
    """Device bytes of one server handle (library + scratch for a chunk)."""
    return lib().linmin_server_handle_bytes(int(L), int(P), int(chunk_pixels), int(host_io))


def linmin_server_destroy(s) -> int:
    return lib().linmin_server_destroy(s)


class Server:
    """Owner of a linmin server; keeps every request's arrays alive until
    its ticket is waited on (the C side reads and writes them meanwhile)."""

    def __init__(self, hbm_budget_bytes: int | None = None, slots: int | None = None,
                 chunk_pixels: int | None = None, max_iter: int | None = None,
                 autotune: bool | None = None):
        o = linmin_server_default_options()
        if autotune is not None:
            o.autotune = int(bool(autotune))
        if hbm_budget_bytes is not None:
            o.hbm_budget_bytes = int(hbm_budget_bytes)
        if slots is not None:
            o.slots = int(slots)
        if chunk_pixels is not None:
            o.chunk_pixels = int(chunk_pixels)
        if max_iter is not None:
            o.max_iter = int(max_iter)
        self.s = linmin_server_create(o)
        self._keep = {}

    def submit(self, library, cube, sigma, abundances=None, uncertainties=None,
               residual_rms=None, iterations=None) -> int:
        P, L = library.shape
        N = cube.shape[0]
        t = linmin_server_submit(self.s, library, L, P, cube, N, sigma, abundances,
                                 uncertainties, residual_rms, iterations)
        self._keep[t] = (library, cube, sigma, abundances, uncertainties, residual_rms,
                         iterations)
        return t

    def poll(self, ticket: int) -> bool:
        return linmin_server_poll(self.s, ticket)

    def wait(self, ticket: int) -> tuple[int, float]:
        st, ms = linmin_server_wait(self.s, ticket)
        self._keep.pop(ticket, None)
        return st, ms

    def stats(self) -> dict:
        return linmin_server_get_stats(self.s)

    def close(self):
        if self.s:
            linmin_server_destroy(self.s)
            self.s = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

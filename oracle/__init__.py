"""FP64 CPU oracle for LinMin's fully constrained unmixing (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product (the CUDA library and its binding)
never does, and shares no code with it: the oracle is the plain C file
``linmin_oracle.c`` compiled by gcc, wrapped here with ctypes.

Functions follow the paper's method (Sec. 2.1-2.3) as documented in the C
source: whitening by the per-band noise, the FCLS problem (x >= 0,
sum x = 1) solved by a Mehrotra primal-dual interior-point method on the
bordered KKT system, the support-restricted estimator covariance as the
abundance uncertainty, and the unwhitened RMS of the fit.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "linmin_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblinmin_oracle.so")
_lib = None
_lock = threading.Lock()

OR_OK, OR_MAXITER, OR_SINGULAR = 0, 1, 2
MAX_ITER = 200


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags, no -march)."""
    os.makedirs(_BUILD, exist_ok=True)
    stamp = os.path.join(_BUILD, "machine")
    same_machine = os.path.exists(stamp) and open(stamp).read() == platform.machine()
    if force or not same_machine or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
        with open(stamp, "w") as f:
            f.write(platform.machine())
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            F = ctypes.POINTER(ctypes.c_float)
            I = ctypes.POINTER(ctypes.c_int)
            lib.oracle_prep.argtypes = [ctypes.c_int, ctypes.c_int, F, F, D, D]
            lib.oracle_project.argtypes = [ctypes.c_int, ctypes.c_int, D, F, F, D, D]
            lib.oracle_project.restype = None
            lib.oracle_fcls.argtypes = [ctypes.c_int, D, D, ctypes.c_double,
                                        ctypes.c_int, D, D, D, I, D]
            lib.oracle_support.argtypes = [ctypes.c_int, D, D, D, I]
            lib.oracle_sigma_x.argtypes = [ctypes.c_int, D, I, D]
            lib.oracle_rms.argtypes = [ctypes.c_int, ctypes.c_int, F, D, F]
            lib.oracle_rms.restype = ctypes.c_double
            lib.oracle_nproc.argtypes = []
            lib.oracle_unmix.argtypes = [ctypes.c_int, ctypes.c_int, F, F,
                                         ctypes.c_longlong, F, ctypes.c_int,
                                         ctypes.c_int, D, D, D, I, D, D, D, I, I]
            lib.oracle_unmix_set.argtypes = [ctypes.c_int, ctypes.c_int, F, F,
                                             ctypes.c_longlong, F, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, D, D, D, I, D, D, D, I, I, D, D]
            lib.oracle_pos.argtypes = [ctypes.c_int, D, D, ctypes.c_double, ctypes.c_int,
                                       D, D, I, D]
            lib.oracle_slo.argtypes = [ctypes.c_int, D, D, ctypes.c_double, ctypes.c_int,
                                       D, D, D, D, I, D]
            lib.oracle_sigma_x_set.argtypes = [ctypes.c_int, D, I, ctypes.c_int, D]
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def nproc() -> int:
    return int(_load().oracle_nproc())


def prep(S, sigma):
    """Whitened Gram G = S W^2 S^T (P x P) and B = W^2 S (P x L), fp64."""
    S, sigma = _f32(S), _f32(sigma)
    P, L = S.shape
    G = np.empty((P, P)); B = np.empty((P, L))
    rc = _load().oracle_prep(L, P, _p(S, ctypes.c_float), _p(sigma, ctypes.c_float),
                             _p(G, ctypes.c_double), _p(B, ctypes.c_double))
    if rc:
        raise ValueError(f"oracle_prep: invalid input (code {rc})")
    return G, B


def project(B, sigma, y):
    """c = B y and s = y^T W^2 y for one pixel."""
    B, sigma, y = _f64(B), _f32(sigma), _f32(y)
    P, L = B.shape
    c = np.empty(P); s = ctypes.c_double()
    _load().oracle_project(L, P, _p(B, ctypes.c_double), _p(sigma, ctypes.c_float),
                           _p(y, ctypes.c_float), _p(c, ctypes.c_double),
                           ctypes.byref(s))
    return c, s.value


def fcls(G, c, s=0.0, max_iter=MAX_ITER):
    """One FCLS problem min 1/2 x'Gx - c'x + s/2, x >= 0, 1'x = 1.

    Returns dict(x, lam, nu, iters, mu, status)."""
    G, c = _f64(G), _f64(c)
    P = c.shape[0]
    x = np.empty(P); lam = np.empty(P)
    nu = ctypes.c_double(); mu = ctypes.c_double(); it = ctypes.c_int()
    st = _load().oracle_fcls(P, _p(G, ctypes.c_double), _p(c, ctypes.c_double),
                             float(s), int(max_iter), _p(x, ctypes.c_double),
                             _p(lam, ctypes.c_double), ctypes.byref(nu),
                             ctypes.byref(it), ctypes.byref(mu))
    return dict(x=x, lam=lam, nu=nu.value, iters=it.value, mu=mu.value, status=st)


def support(G, x, lam):
    G, x, lam = _f64(G), _f64(x), _f64(lam)
    P = x.shape[0]
    m = np.empty(P, dtype=np.int32)
    _load().oracle_support(P, _p(G, ctypes.c_double), _p(x, ctypes.c_double),
                           _p(lam, ctypes.c_double), _p(m, ctypes.c_int))
    return m.astype(bool)


def sigma_x(G, in_S):
    G = _f64(G)
    m = np.ascontiguousarray(in_S, dtype=np.int32)
    P = m.shape[0]
    sx = np.empty(P)
    _load().oracle_sigma_x(P, _p(G, ctypes.c_double), _p(m, ctypes.c_int),
                           _p(sx, ctypes.c_double))
    return sx


def rms(S, x, y):
    S, x, y = _f32(S), _f64(x), _f32(y)
    P, L = S.shape
    return float(_load().oracle_rms(L, P, _p(S, ctypes.c_float), _p(x, ctypes.c_double),
                                    _p(y, ctypes.c_float)))


def unmix(S, sigma, X, nthreads: int = 0, max_iter: int = MAX_ITER,
          extras: bool = True):
    """Unmix every pixel of X (N x L) against S (P x L) on ``nthreads`` cores.

    Returns dict with x, sx (N x P), rms, iters (N, negative = not
    converged) and, when ``extras``, lam (N x P), nu, mu, status, ksup (N)."""
    S, sigma, X = _f32(S), _f32(sigma), _f32(X)
    P, L = S.shape
    N = X.shape[0]
    if X.shape[1] != L or sigma.shape[0] != L:
        raise ValueError("shape mismatch between S, sigma and X")
    out = dict(x=np.empty((N, P)), sx=np.empty((N, P)), rms=np.empty(N),
               iters=np.empty(N, dtype=np.int32))
    if extras:
        out.update(lam=np.empty((N, P)), nu=np.empty(N), mu=np.empty(N),
                   status=np.empty(N, dtype=np.int32),
                   ksup=np.empty(N, dtype=np.int32))
    D, I = ctypes.c_double, ctypes.c_int

    def opt(k, t):
        return _p(out[k], t) if k in out else None

    rc = _load().oracle_unmix(L, P, _p(S, ctypes.c_float), _p(sigma, ctypes.c_float),
                              N, _p(X, ctypes.c_float), int(max_iter), int(nthreads),
                              _p(out["x"], D), _p(out["sx"], D), _p(out["rms"], D),
                              _p(out["iters"], I), opt("lam", D), opt("nu", D),
                              opt("mu", D), opt("status", I), opt("ksup", I))
    if rc:
        raise ValueError(f"oracle_unmix: invalid input (code {rc})")
    return out


CONSTRAINTS = {"sto": 0, "slo": 1, "pos": 2}


def unmix_constraint(S, sigma, X, constraint: str = "sto", max_iter: int = MAX_ITER,
                     nthreads: int = 0):
    """Unmixing under the constraint sets of the paper (Sec. 2.2 and the runs
    of Sec. 4): "sto" x >= 0, sum x = 1 (``unmix``); "slo" x >= 0,
    sum x <= 1 (``oracle_slo``: the inequality with its slack w and
    multiplier omega); "pos" x >= 0 alone (``oracle_pos``: no bound on the
    sum).  The uncertainty is the support-restricted inverse Hessian,
    bordered by the sum constraint only where it is active (slo: omega > w).

    Returns dict(x, sx, rms, iters, lam) like ``unmix``, plus for slo the
    slack w (= 1 - sum x) and its multiplier omega."""
    if constraint not in CONSTRAINTS:
        raise ValueError("constraint must be sto, slo or pos")
    if constraint == "sto":
        return unmix(S, sigma, X, max_iter=max_iter, nthreads=nthreads)
    S, sigma, X = _f32(S), _f32(sigma), _f32(X)
    P, L = S.shape
    N = X.shape[0]
    if X.shape[1] != L or sigma.shape[0] != L:
        raise ValueError("shape mismatch between S, sigma and X")
    out = dict(x=np.empty((N, P)), sx=np.empty((N, P)), rms=np.empty(N),
               iters=np.empty(N, dtype=np.int32), lam=np.empty((N, P)),
               slack=np.empty(N), omega=np.empty(N))
    D, I = ctypes.c_double, ctypes.c_int
    rc = _load().oracle_unmix_set(L, P, _p(S, ctypes.c_float), _p(sigma, ctypes.c_float),
                                  N, _p(X, ctypes.c_float), CONSTRAINTS[constraint],
                                  int(max_iter), int(nthreads), _p(out["x"], D),
                                  _p(out["sx"], D), _p(out["rms"], D), _p(out["iters"], I),
                                  _p(out["lam"], D), None, None, None, None,
                                  _p(out["slack"], D), _p(out["omega"], D))
    if rc:
        raise ValueError(f"oracle_unmix_set: invalid input (code {rc})")
    if constraint == "pos":
        del out["slack"], out["omega"]
    return out


def pos(G, c, s=0.0, max_iter=MAX_ITER):
    """One pos problem min 1/2 x'Gx - c'x + s/2, x >= 0."""
    G, c = _f64(G), _f64(c)
    P = c.shape[0]
    x = np.empty(P); lam = np.empty(P); it = ctypes.c_int(); mu = ctypes.c_double()
    st = _load().oracle_pos(P, _p(G, ctypes.c_double), _p(c, ctypes.c_double), float(s),
                            int(max_iter), _p(x, ctypes.c_double), _p(lam, ctypes.c_double),
                            ctypes.byref(it), ctypes.byref(mu))
    return dict(x=x, lam=lam, iters=it.value, mu=mu.value, status=st)


def slo(G, c, s=0.0, max_iter=MAX_ITER):
    """One slo problem min 1/2 x'Gx - c'x + s/2, x >= 0, 1'x <= 1."""
    G, c = _f64(G), _f64(c)
    P = c.shape[0]
    x = np.empty(P); lam = np.empty(P); w = ctypes.c_double(); om = ctypes.c_double()
    it = ctypes.c_int(); mu = ctypes.c_double()
    st = _load().oracle_slo(P, _p(G, ctypes.c_double), _p(c, ctypes.c_double), float(s),
                            int(max_iter), _p(x, ctypes.c_double), _p(lam, ctypes.c_double),
                            ctypes.byref(w), ctypes.byref(om), ctypes.byref(it),
                            ctypes.byref(mu))
    return dict(x=x, lam=lam, w=w.value, omega=om.value, iters=it.value, mu=mu.value,
                status=st)


def sigma_x_set(G, in_S, bordered: bool):
    G = _f64(G)
    m = np.ascontiguousarray(in_S, dtype=np.int32)
    P = m.shape[0]
    sx = np.empty(P)
    _load().oracle_sigma_x_set(P, _p(G, ctypes.c_double), _p(m, ctypes.c_int), int(bordered),
                               _p(sx, ctypes.c_double))
    return sx


def unmix_cov(S, cov_inv, X, max_iter: int = MAX_ITER):
    """Unmixing under a full noise covariance C (Sec. 2.3, eq.
    RenormalizedProblem: the data are whitened as X' = X L with
    C^-1 = L L^T).  The whitened criterion ||L^T (y - S^T x)||^2 has the
    Gram G = S C^-1 S^T and the projection c = S C^-1 y; each pixel is then
    the same fully constrained problem as with a diagonal C, solved by
    ``fcls`` (fp64), with the uncertainty of ``sigma_x`` on the support of
    ``support`` and the unwhitened RMS of ``rms``.  G and c are formed in
    fp64 (numpy); there is no per-band sigma.

    Returns dict(x, sx, rms, iters, lam) like ``unmix``, and the Gram G."""
    S32, X32 = _f32(S), _f32(X)
    S64, X64 = S32.astype(np.float64), X32.astype(np.float64)
    Ci = np.asarray(cov_inv, dtype=np.float64)
    P, L = S64.shape
    if Ci.shape != (L, L) or X64.shape[1] != L:
        raise ValueError("shape mismatch between S, cov_inv and X")
    T = Ci @ S64.T                 # L x P
    G = S64 @ T                    # S C^-1 S^T
    Cp = X64 @ T                   # rows: c = S C^-1 y
    sy = np.einsum("nl,lm,nm->n", X64, Ci, X64)
    N = X64.shape[0]
    out = dict(x=np.empty((N, P)), sx=np.empty((N, P)), rms=np.empty(N),
               iters=np.empty(N, dtype=np.int32), lam=np.empty((N, P)), G=G)
    for n in range(N):
        r = fcls(G, Cp[n], sy[n], max_iter)
        out["lam"][n] = r["lam"]
        x = np.maximum(r["x"], 0.0)
        x /= x.sum()
        m = support(G, r["x"], r["lam"])
        out["x"][n] = x
        out["sx"][n] = sigma_x(G, m)
        out["rms"][n] = rms(S32, x, X32[n])
        out["iters"][n] = r["iters"] if r["status"] == OR_OK else -r["iters"]
    return out


def objective(G, c, s, x):
    """f(x) = 1/2 x'Gx - c'x + s/2 in fp64 (the whitened half squared error)."""
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * x @ G @ x - c @ x + 0.5 * s

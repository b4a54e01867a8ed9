"""Detection products, plain numpy (test infrastructure, like the rest of
``oracle``): only the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may use it; the CUDA library shares no code with it.

* ``paper_extra_spectra``: the additional spectra of Sec. 2.5 and the
  Appendix table (names 33-44).
* ``detect``: the detection conditions of Sec. 4 (introduction), evaluated
  pixel by pixel in float32 like the values they compare, with per-mineral
  counts, sums, arg-max and, given the truth, the positive / false
  detection counts of Sec. 3.1.
* ``threshold_sums`` and ``thresholds``: eq. Threshold of Sec. 3.1.
* ``second_pass``: the second unmixing of Sec. 5 with the detected spectra
  only, per pixel.
"""
from __future__ import annotations

import math

import numpy as np


def paper_extra_spectra(L: int, wavelengths=None, n_extras: int = 12) -> np.ndarray:
    """Rows: Flat 1, Flat 0.0001, slope increasing, slope decreasing, then
    cos, sin, -cos, -sin with a quarter period over the domain ("1/4") and
    with half a period ("1/2"), over u = (w - w_0) / (w_{L-1} - w_0) in
    [0, 1] (evenly spaced when ``wavelengths`` is None).  fp64."""
    if n_extras not in (4, 12) or L < 2:
        raise ValueError("n_extras must be 4 or 12 and L >= 2")
    if wavelengths is None:
        u = np.arange(L, dtype=np.float64) / (L - 1)
    else:
        w = np.asarray(wavelengths, dtype=np.float32).astype(np.float64)
        u = (w - w[0]) / (w[-1] - w[0])
    rows = [np.ones(L), np.full(L, 1e-4), u, 1.0 - u]
    for quarter_periods in (1, 2):          # argument pi/2 * u, then pi * u
        t = 0.5 * math.pi * quarter_periods * u
        rows += [np.cos(t), np.sin(t), -np.cos(t), -np.sin(t)]
    return np.stack(rows[:n_extras])


def detect(x, sx=None, rms=None, iterations=None, truth=None, x_min=None,
           rms_max: float = np.inf, n_minerals: int | None = None) -> dict:
    """Mineral i < n_minerals is detected in pixel n when x[n, i] > x_min[i]
    (above the mineral's threshold), sx[n, i] < x[n, i] (the uncertainty
    below the abundance) and rms[n] < rms_max (the fit within the noise);
    a missing array drops its condition, and a pixel with iterations < 0
    detects nothing.  Comparisons are of float32 values.

    Returns dict(mask (N uint64, bit i = detected), count, xsum (fp64),
    xmax, argmax (smallest pixel of the largest detected x_i, -1 if none),
    n_true, true_pos, false_pos)."""
    x = np.asarray(x, dtype=np.float32)
    N, P = x.shape
    nm = P if n_minerals is None else int(n_minerals)
    ok = np.ones(N, dtype=bool)
    if rms is not None:
        ok &= np.asarray(rms, dtype=np.float32) < np.float32(rms_max)
    if iterations is not None:
        ok &= np.asarray(iterations) >= 0
    xm = np.asarray(x_min, dtype=np.float32)[:nm] if nm else np.zeros(0, np.float32)
    det = np.zeros((N, P), dtype=bool)
    for i in range(nm):
        d = x[:, i] > xm[i]
        if sx is not None:
            d &= np.asarray(sx, dtype=np.float32)[:, i] < x[:, i]
        det[:, i] = d & ok
    mask = np.zeros(N, dtype=np.uint64)
    for i in range(nm):
        mask |= det[:, i].astype(np.uint64) << np.uint64(i)
    out = dict(mask=mask, count=np.zeros(P, np.int64), xsum=np.zeros(P),
               xmax=np.zeros(P, np.float32), argmax=np.full(P, -1, np.int64),
               n_true=np.zeros(P, np.int64), true_pos=np.zeros(P, np.int64),
               false_pos=np.zeros(P, np.int64))
    tr = None
    if truth is not None:
        t = np.asarray(truth, dtype=np.uint64)
        tr = np.stack([((t >> np.uint64(i)) & np.uint64(1)).astype(bool) for i in range(P)], 1) \
            if N else np.zeros((0, P), dtype=bool)
    for i in range(nm):
        idx = np.nonzero(det[:, i])[0]
        out["count"][i] = idx.size
        if idx.size:
            v = x[idx, i]
            out["xsum"][i] = float(np.sum(v.astype(np.float64)))
            out["xmax"][i] = v.max()
            out["argmax"][i] = idx[np.argmax(v)]       # first occurrence of the maximum
        if tr is not None:
            out["n_true"][i] = int(tr[:, i].sum())
            out["true_pos"][i] = int((det[:, i] & tr[:, i]).sum())
            out["false_pos"][i] = int((det[:, i] & ~tr[:, i]).sum())
    return out


def threshold_sums(x, truth, n_minerals: int) -> dict:
    """Counts, sums and sums of squared deviations from the mean (fp64) of
    x[:, i] over the pixels where mineral i is present (pos) and absent
    (neg)."""
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    t = np.asarray(truth, dtype=np.uint64)
    P = x.shape[1]
    keys = ("n_pos", "n_neg", "sum_pos", "m2_pos", "sum_neg", "m2_neg")
    out = {k: np.zeros(P, np.int64 if k.startswith("n_") else np.float64) for k in keys}
    for i in range(n_minerals):
        pres = ((t >> np.uint64(i)) & np.uint64(1)).astype(bool)
        for name, sel in (("pos", pres), ("neg", ~pres)):
            v = x[sel, i]
            out["n_" + name][i] = v.size
            out["sum_" + name][i] = v.sum()
            out["m2_" + name][i] = ((v - v.mean()) ** 2).sum() if v.size else 0.0
    return out


def thresholds(x, truth, n_minerals: int) -> np.ndarray:
    """eq. Threshold: C_i = 1/2 (mean(A_pos) - 2 std(A_pos) + mean(A_false)
    + 6 std(A_false)) over the estimated abundances of the pixels where
    mineral i is present (pos) and absent (false); population standard
    deviations.  NaN when either set is empty."""
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    t = np.asarray(truth, dtype=np.uint64)
    C = np.full(n_minerals, np.nan)
    for i in range(n_minerals):
        pres = ((t >> np.uint64(i)) & np.uint64(1)).astype(bool)
        a_pos, a_false = x[pres, i], x[~pres, i]
        if a_pos.size and a_false.size:
            C[i] = 0.5 * (a_pos.mean() - 2.0 * a_pos.std() + a_false.mean() + 6.0 * a_false.std())
    return C


def second_pass(S, sigma, X, mask, n_minerals: int) -> dict:
    """The second pass of Sec. 5: every pixel unmixed again with only the
    minerals detected in it (bits of ``mask`` below n_minerals) and all the
    additional spectra (columns >= n_minerals), with the sum-to-one oracle
    ``oracle.unmix``.  Abundances and uncertainties of the left-out
    columns are 0.  Returns dict(x, sx, lam (N x P: the multipliers of
    x >= 0, 0 off the kept columns), rms, iters (N))."""
    from . import unmix
    S = np.asarray(S, dtype=np.float32)
    X = np.asarray(X, dtype=np.float32)
    P = S.shape[0]
    N = X.shape[0]
    if not 0 <= n_minerals < P:
        raise ValueError("0 <= n_minerals < P: the additional spectra are always kept")
    keep = np.uint64((1 << n_minerals) - 1)
    m = np.asarray(mask, dtype=np.uint64) & keep
    out = dict(x=np.zeros((N, P)), sx=np.zeros((N, P)), lam=np.zeros((N, P)), rms=np.zeros(N),
               iters=np.zeros(N, np.int32))
    for key in np.unique(m):
        rows = np.nonzero(m == key)[0]
        cols = [i for i in range(n_minerals) if (int(key) >> i) & 1] + list(range(n_minerals, P))
        r = unmix(S[cols], sigma, X[rows])
        out["x"][np.ix_(rows, cols)] = r["x"]
        out["sx"][np.ix_(rows, cols)] = r["sx"]
        out["lam"][np.ix_(rows, cols)] = r["lam"]
        out["rms"][rows] = r["rms"]
        out["iters"][rows] = r["iters"]
    return out

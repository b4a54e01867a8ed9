"""Seeded synthetic hyperspectral workloads for the FCLS unmixing path.

This module only *draws inputs*: a reference library S (one spectrum per
row), per-band noise standard deviations sigma, true abundances and the
observed cube X = A_true . S + E of the linear mixing model (Sec. 2.1,
eq. LinearMixing).  It holds none of the unmixing arithmetic (no whitening,
no Gram matrix, no solver), so both the FP64 CPU oracle and the CUDA path
consume it without sharing any of the method's code.

The paper's real inputs (the USGS/CAT mineral spectra of the Appendix table,
the OMEGA ORB422_4, CRISM frt0000A09C and M3 cubes of Sec. 4) are not
available, so smooth synthetic stand-ins with the same shapes are drawn:

* wavelength grid lambda = linspace(1.0, 2.5, L) micrometres;
* a mineral = quadratic continuum rescaled into [0.2, 0.6], times 1 to 4
  Gaussian absorption bands (depth U[0.05, 0.3], FWHM U[10, 60] nm,
  centre U[1.0, 2.5] um);
* the four additional spectra of Sec. 2.5 (level and slope terms): an
  aerosol-like smooth decay 0.3*exp(-(lambda-1)/0.8), the increasing slope u,
  a decreasing slope 0.5*(1-u) and the constant 1, with
  u = (lambda - lambda_min)/(lambda_max - lambda_min);
* abundances: k active minerals (k uniform in 1..kmax), Dirichlet(0.3) on
  them, extras 0 in the truth;
* noise: N(0, sigma_l^2), sigma_l either constant or U[0.002, 0.02] per band.

All arrays come out as float32 in the layouts the C ABI takes:
``S`` (P, L) row-major == the L x P column-major library,
``X`` (N, L) row-major == the pixel-major (BIP) cube.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BASE_SEED = 20140218
EXTRA_NAMES = ("aerosol_slope", "slope_increasing", "slope_decreasing", "flat_1")


@dataclasses.dataclass(frozen=True)
class CubeSpec:
    """Shape and draw recipe of one synthetic cube."""
    name: str
    n_pix: int
    L: int
    n_minerals: int
    n_extras: int = 0          # 0 or 4 (Sec. 2.5 level/slope spectra)
    n_near_dup: int = 0        # minerals that are perturbed copies of others
    kmax: int = 3              # active minerals per pixel: uniform 1..kmax
    pure_frac: float = 0.0     # fraction of pixels forced to k = 1
    sigma_const: float | None = None   # constant per-band noise, else U[lo, hi]
    sigma_lo: float = 0.002
    sigma_hi: float = 0.02
    seed: int = BASE_SEED
    shape: tuple | None = None  # (lines, samples) of the image, informative

    @property
    def P(self) -> int:
        return self.n_minerals + self.n_extras


# The five workloads.  Index i uses seed BASE_SEED + i.
FCLS_1K = CubeSpec("fcls_1k_L128_P32", 1000, 128, 32, 0, sigma_const=0.005,
                   seed=BASE_SEED + 0, shape=(40, 25))
OMEGA_262K = CubeSpec("omega_262k_L184_P36", 262144, 184, 32, 4,
                      seed=BASE_SEED + 1, shape=(128, 2048))
CRISM_307K = CubeSpec("crism_307k_L240_P48", 307200, 240, 44, 4, n_near_dup=8,
                      kmax=5, pure_frac=0.05, seed=BASE_SEED + 2,
                      shape=(640, 480))
WORKLOADS = (FCLS_1K, OMEGA_262K, CRISM_307K)


def wavelengths(L: int) -> np.ndarray:
    return np.linspace(1.0, 2.5, L)


def _mineral(rng: np.random.Generator, lam: np.ndarray) -> np.ndarray:
    u = (lam - lam[0]) / (lam[-1] - lam[0])
    a, b, c = rng.uniform(-1.0, 1.0, size=3)
    poly = a + b * u + c * u * u
    lo, hi = np.sort(rng.uniform(0.2, 0.6, size=2))
    if hi - lo < 0.02:
        hi = min(0.6, lo + 0.02)
    span = poly.max() - poly.min()
    cont = lo + (hi - lo) * (poly - poly.min()) / span if span > 0 else np.full_like(u, lo)
    spec = cont.copy()
    for _ in range(int(rng.integers(1, 5))):
        depth = rng.uniform(0.05, 0.3)
        fwhm = rng.uniform(0.010, 0.060)
        s = fwhm / 2.3548
        centre = rng.uniform(1.0, 2.5)
        spec *= 1.0 - depth * np.exp(-((lam - centre) ** 2) / (2.0 * s * s))
    return spec


def extra_spectra(L: int) -> np.ndarray:
    """The four level/slope spectra of Sec. 2.5 (rows), fp64."""
    lam = wavelengths(L)
    u = (lam - lam[0]) / (lam[-1] - lam[0])
    return np.stack([0.3 * np.exp(-(lam - 1.0) / 0.8), u, 0.5 * (1.0 - u),
                     np.ones(L)])


def library(rng: np.random.Generator, L: int, n_minerals: int, n_extras: int,
            n_near_dup: int = 0) -> np.ndarray:
    """Library S, shape (P, L) fp64: minerals first, then the extras."""
    lam = wavelengths(L)
    n_orig = n_minerals - n_near_dup
    rows = [_mineral(rng, lam) for _ in range(n_orig)]
    for _ in range(n_near_dup):
        src = rows[int(rng.integers(0, n_orig))]
        rows.append(src * (1.0 + rng.normal(0.0, 0.01, size=L)))
    S = np.stack(rows)
    if n_extras:
        if n_extras != 4:
            raise ValueError("only the 4 level/slope extras are drawn")
        S = np.concatenate([S, extra_spectra(L)])
    return S


def check_unique(S: np.ndarray) -> bool:
    """True when rank [S^T; 1^T] = P, the condition for a unique FCLS minimiser."""
    P = S.shape[0]
    M = np.concatenate([S.T.astype(np.float64), np.ones((1, P))])
    return int(np.linalg.matrix_rank(M)) == P


def abundances(rng: np.random.Generator, n_pix: int, P: int, n_minerals: int,
               kmax: int, pure_frac: float = 0.0) -> np.ndarray:
    """True abundances (n_pix, P) fp64 on the simplex; extras are 0."""
    k = rng.integers(1, kmax + 1, size=n_pix)
    if pure_frac > 0:
        k[rng.random(n_pix) < pure_frac] = 1
    idx = np.argsort(rng.random((n_pix, n_minerals)), axis=1)[:, :kmax]
    g = rng.gamma(0.3, 1.0, size=(n_pix, kmax))
    g[np.arange(kmax)[None, :] >= k[:, None]] = 0.0
    # a pixel whose draws all underflow to 0 becomes pure in its first pick
    dead = g.sum(axis=1) <= 0
    g[dead, 0] = 1.0
    g /= g.sum(axis=1, keepdims=True)
    x = np.zeros((n_pix, P))
    np.put_along_axis(x, idx, g, axis=1)
    return x


def noise_sigma(rng: np.random.Generator, spec: CubeSpec) -> np.ndarray:
    if spec.sigma_const is not None:
        return np.full(spec.L, spec.sigma_const)
    return rng.uniform(spec.sigma_lo, spec.sigma_hi, size=spec.L)


@dataclasses.dataclass
class Cube:
    spec: CubeSpec
    S: np.ndarray        # (P, L) float32 library, row j = spectrum j
    sigma: np.ndarray    # (L,) float32 per-band noise std
    X: np.ndarray        # (N, L) float32 observed spectra, pixel-major
    A_true: np.ndarray   # (N, P) float64 abundances that generated X

    @property
    def N(self) -> int:
        return self.X.shape[0]

    @property
    def L(self) -> int:
        return self.X.shape[1]

    @property
    def P(self) -> int:
        return self.S.shape[0]


def make_cube(spec: CubeSpec, n_pix: int | None = None) -> Cube:
    """Draw the cube of ``spec``; ``n_pix`` truncates to its first pixels.

    The library and sigma do not depend on ``n_pix``; the first ``n_pix``
    pixels of a truncated cube are the same as those of the full cube.
    """
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    S = library(rng, spec.L, spec.n_minerals, spec.n_extras, spec.n_near_dup)
    if not check_unique(S):
        raise RuntimeError(f"{spec.name}: rank [S^T; 1^T] < P, minimiser not unique")
    sigma = noise_sigma(rng, spec)
    N = spec.n_pix if n_pix is None else min(int(n_pix), spec.n_pix)
    # pixel draws come from a child stream so truncation keeps a prefix
    prng = np.random.Generator(np.random.PCG64(spec.seed + 7919))
    A = abundances(prng, spec.n_pix, spec.P, spec.n_minerals, spec.kmax,
                   spec.pure_frac)[:N]
    nrng = np.random.Generator(np.random.PCG64(spec.seed + 104729))
    X = np.empty((N, spec.L), dtype=np.float32)
    S32 = S.astype(np.float32)
    chunk = 65536
    for lo in range(0, N, chunk):
        hi = min(N, lo + chunk)
        E = nrng.standard_normal((hi - lo, spec.L)) * sigma[None, :]
        X[lo:hi] = (A[lo:hi] @ S + E).astype(np.float32)
    return Cube(spec, S32, sigma.astype(np.float32), X, A)


def random_instance(seed: int, N: int, L: int, P: int, n_extras: int = 0,
                    kmax: int = 3, sigma_const: float | None = None,
                    n_near_dup: int = 0, pure_frac: float = 0.0) -> Cube:
    """A small cube of arbitrary shape (tests: tiny P, ragged N, ...)."""
    spec = CubeSpec(f"rand_{seed}_{N}x{L}x{P}", N, L, P - n_extras, n_extras,
                    n_near_dup=n_near_dup, kmax=min(kmax, P - n_extras),
                    pure_frac=pure_frac, sigma_const=sigma_const, seed=seed)
    return make_cube(spec)


# ---------------------------------------------------------------- batches
BATCH_L = (128, 184, 240)
BATCH_P = (16, 32, 48, 64)


def batch_specs(n_cubes: int = 64, seed: int = BASE_SEED + 3,
                n_min: float = 1e3, n_max: float = 3e5) -> list[CubeSpec]:
    """Uneven cubes: N log-uniform in [n_min, n_max], L and P drawn from sets."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n_cubes):
        N = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        L = int(rng.choice(BATCH_L))
        P = int(rng.choice(BATCH_P))
        out.append(CubeSpec(f"batch{i}_N{N}_L{L}_P{P}", N, L, P - 4, 4,
                            seed=seed * 1000 + i))
    return out


def poisson_arrivals(n: int, rate_per_s: float = 200.0,
                     seed: int = BASE_SEED + 4) -> np.ndarray:
    """Arrival times (s) of a Poisson stream of ``n`` requests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


# ------------------------------------------------------ full covariance
def ar1_covariance(sigma: np.ndarray, rho: float) -> np.ndarray:
    """C = D R D with D = diag(sigma) and R_lm = rho^|l - m|: noise whose
    neighbouring bands are correlated (the off-diagonal terms of Sec. 2.3),
    L x L float64."""
    sg = np.asarray(sigma, dtype=np.float64)
    idx = np.arange(sg.shape[0])
    R = float(rho) ** np.abs(idx[:, None] - idx[None, :])
    return sg[:, None] * R * sg[None, :]


def make_cube_cov(spec: CubeSpec, rho: float, n_pix: int | None = None):
    """The cube of ``spec`` (same library, sigma and abundances) with noise
    drawn from the AR(1) covariance of ``ar1_covariance(sigma, rho)``.
    Returns (cube, C, C^-1)."""
    base = make_cube(spec, n_pix=1)
    S, sigma = base.S.astype(np.float64), base.sigma.astype(np.float64)
    N = spec.n_pix if n_pix is None else min(int(n_pix), spec.n_pix)
    prng = np.random.Generator(np.random.PCG64(spec.seed + 7919))
    A = abundances(prng, spec.n_pix, spec.P, spec.n_minerals, spec.kmax,
                   spec.pure_frac)[:N]
    C = ar1_covariance(sigma, rho)
    Lc = np.linalg.cholesky(C)
    nrng = np.random.Generator(np.random.PCG64(spec.seed + 15485863))
    X = np.empty((N, spec.L), dtype=np.float32)
    for lo in range(0, N, 65536):
        hi = min(N, lo + 65536)
        E = nrng.standard_normal((hi - lo, spec.L)) @ Lc.T
        X[lo:hi] = (A[lo:hi] @ S + E).astype(np.float32)
    Cinv = np.linalg.inv(C)
    Cinv = 0.5 * (Cinv + Cinv.T)
    return Cube(spec, base.S, base.sigma, X, A), C, Cinv


# ------------------------------------------- surface mixtures (Sec. 3.1)
def surface_mixtures(n: int = 1000, L: int = 184, n_ref: int = 32, flat: float = 0.35,
                     frac_max: float = 0.1, noise_mean: float = 1.3e-3,
                     seed: int = BASE_SEED + 5):
    """The synthetic surface of Sec. 3.1: every spectrum is a binary mixture
    of a flat component at reflectance ``flat`` and one of ``n_ref``
    reference spectra (drawn uniformly), with the reference's share a drawn
    uniformly in (0, frac_max): y = (1 - a) flat + a S_i + noise, so that
    each reference is present in about n / n_ref spectra.  The noise is
    N(0, sigma_l^2) with sigma_l uniform in [0.5, 1.5] * noise_mean (a
    wavelength-average standard deviation of noise_mean).

    The library is the n_ref references followed by the four level/slope
    extras of this module (aerosol, u, 0.5 (1 - u), 1); the flat component
    is the sum-to-one combination 0.025 * 1 + 0.325 u + 0.65 * 0.5 (1 - u)
    (level 0.35, sum 1) scaled by (1 - a), so ``A_true`` is on the simplex.

    Returns (cube, truth): truth[n] has bit i set when reference i is
    present in spectrum n (uint64)."""
    if abs(flat - 0.35) > 1e-12:
        raise ValueError("the extras' combination above is worked out for flat = 0.35")
    rng = np.random.Generator(np.random.PCG64(seed))
    S = library(rng, L, n_ref, 4)
    if not check_unique(S):
        raise RuntimeError("surface library: rank [S^T; 1^T] < P")
    sigma = noise_mean * rng.uniform(0.5, 1.5, size=L)
    ref = rng.integers(0, n_ref, size=n)
    a = frac_max * (1.0 - rng.random(n))              # (0, frac_max]
    A = np.zeros((n, n_ref + 4))
    A[np.arange(n), ref] = a
    A[:, n_ref + 1] = 0.325 * (1.0 - a)               # slope increasing u
    A[:, n_ref + 2] = 0.65 * (1.0 - a)                # 0.5 (1 - u)
    A[:, n_ref + 3] = 0.025 * (1.0 - a)               # flat 1
    E = rng.standard_normal((n, L)) * sigma[None, :]
    X = (A @ S + E).astype(np.float32)
    spec = CubeSpec(f"surface_{n}_L{L}_P{n_ref + 4}", n, L, n_ref, 4,
                    sigma_lo=0.5 * noise_mean, sigma_hi=1.5 * noise_mean, seed=seed)
    truth = np.left_shift(np.uint64(1), ref.astype(np.uint64))
    return Cube(spec, S.astype(np.float32), sigma.astype(np.float32), X, A), truth


def truth_masks(A_true: np.ndarray, n_minerals: int) -> np.ndarray:
    """Bit i of entry n set when mineral i < n_minerals has a non-zero true
    abundance in pixel n (uint64)."""
    m = np.zeros(A_true.shape[0], dtype=np.uint64)
    for i in range(n_minerals):
        m |= (A_true[:, i] > 0).astype(np.uint64) << np.uint64(i)
    return m


def detection_inputs(seed: int, N: int, P: int, n_minerals: int, x_min: np.ndarray,
                     rms_max: float):
    """Seeded arrays shaped like unmixing outputs for the detection tests:
    abundances on the simplex, many exactly at or one ulp around a
    threshold, uncertainties equal to or near their abundance, RMS values
    at and around rms_max, a few negative iteration counts, random truth
    masks.  Returns (x, sx, rms, iterations, truth)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.dirichlet(np.full(P, 0.3), size=N).astype(np.float32) if N else np.zeros((0, P), np.float32)
    xm = np.asarray(x_min, dtype=np.float32)
    for i in range(min(n_minerals, P)):           # exact ties and one-ulp neighbours
        sel = rng.random(N) < 0.1
        k = int(sel.sum())
        x[sel, i] = rng.choice(np.array([xm[i], np.nextafter(xm[i], np.float32(1)),
                                         np.nextafter(xm[i], np.float32(0))], np.float32), k)
    sx = (x * rng.uniform(0.3, 1.3, size=x.shape)).astype(np.float32)
    eq = rng.random(x.shape) < 0.05
    sx[eq] = x[eq]
    rms = np.float32(rms_max) * rng.uniform(0.5, 1.5, size=N).astype(np.float32)
    rms[rng.random(N) < 0.05] = np.float32(rms_max)
    it = rng.integers(5, 30, size=N).astype(np.int32)
    it[rng.random(N) < 0.02] *= -1
    truth = rng.integers(0, 2 ** 63, size=N, dtype=np.int64).astype(np.uint64)
    return x, sx, rms.astype(np.float32), it, truth

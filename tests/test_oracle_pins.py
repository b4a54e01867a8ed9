"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle (``oracle/``) against something other than
itself: exhaustive support enumeration (the combination search of Sec. 2.1
reused as a check), the Frank-Wolfe/KKT optimality certificates of the
convex problem of Sec. 2.2, closed forms (P = 1, P = 2, interior SCLS),
exact noise-free mixtures, invariances of the whitened problem of Sec. 2.3,
a Monte-Carlo check of the "error provided by the Hessian" (Sec. 2.3), the
RMS of the fit, and an independent NNLS-based FCLS (scipy).
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from tests import _pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny_library(rng, P, L, with_extras):
    if with_extras and P >= 6:
        S = synth.library(rng, L, P - 4, 4)
    else:
        S = synth.library(rng, L, P, 0)
    return S.astype(np.float32)


@pytest.mark.parametrize("seed", range(24))
def test_brute_force_small_P(seed):
    """x equals the exhaustive-support minimiser; sigma_x equals the bordered
    inverse on that support."""
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    P = int(rng.integers(2, 11))
    L = int(rng.integers(P + 2, 4 * P + 8))
    S = _tiny_library(rng, P, L, with_extras=seed % 2 == 0)
    if not synth.check_unique(S):
        pytest.skip("drawn library not unique")
    sigma = rng.uniform(0.002, 0.02, size=L).astype(np.float32)
    N = 4
    xt = synth.abundances(rng, N, P, P, min(3, P))
    X = (xt @ S.astype(np.float64) + rng.standard_normal((N, L)) * sigma).astype(np.float32)
    r = oracle.unmix(S, sigma, X, nthreads=1)
    assert np.all(r["iters"] >= 0)
    for n in range(N):
        G, c, s = _pins.qp_terms(S, sigma, X[n])
        xb = _pins.brute_force(G, c, s)
        np.testing.assert_allclose(r["x"][n], xb, atol=2e-8, rtol=0)
        f_or = _pins.objective(G, c, s, r["x"][n])
        f_bf = _pins.objective(G, c, s, xb)
        assert f_or - f_bf <= 1e-9 * max(1.0, abs(f_bf))
        idx = np.flatnonzero(xb > 1e-9)
        lam = r["lam"][n]
        # strictly complementary pixels only: the support is then unambiguous
        ratio = lam / np.maximum(r["x"][n], 1e-300) / np.diag(G)
        if np.all((ratio < 1e-4) | (ratio > 1e4)):
            np.testing.assert_allclose(r["sx"][n], _pins.support_sigma(G, idx),
                                       rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("spec", synth.WORKLOADS, ids=lambda s: s.name)
def test_kkt_certificate_on_workloads(spec):
    """Feasible, Frank-Wolfe gap ~ 0 and KKT conditions on sampled pixels."""
    cube = synth.make_cube(spec, n_pix=400)
    r = oracle.unmix(cube.S, cube.sigma, cube.X)
    assert np.all(r["iters"] >= 0), "oracle hit its iteration cap"
    G, B = _pins.whiten(cube.S, cube.sigma)
    scale = np.max(np.diag(G))
    for n in range(cube.N):
        x = r["x"][n]
        c = B @ cube.X[n].astype(np.float64)
        assert abs(x.sum() - 1.0) <= 1e-12
        assert x.min() >= 0.0
        gap = _pins.fw_gap(G, c, x)
        assert gap <= 1e-9 * scale, gap
        stat, dual = _pins.kkt_violation(G, c, x, support_tol=1e-9)
        assert stat <= 1e-6 * scale and dual <= 1e-6 * scale


def test_golden_exact_mixtures():
    """Noise-free dyadic mixtures (exact in fp32) are recovered to 1e-10.

    Where x has zeros the problem is degenerate (zero residual makes the
    multiplier of every inactive coordinate zero as well): an interior-point
    iterate then approaches x_i = lambda_i = 0 at the rate sqrt(mu), and the
    stopping rule mu <= 1e-13 (1 + |f|) bounds the error by ~3e-7; 1e-8 is
    asserted there."""
    with open(os.path.join(GOLDEN, "dyadic_mixtures.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        S = (np.array(case["S_num"], dtype=np.float64) / case["S_den"]).astype(np.float32)
        x = np.array(case["x"])
        y64 = x @ S.astype(np.float64)
        y = y64.astype(np.float32)
        assert np.array_equal(y.astype(np.float64), y64), "fixture not exact in fp32"
        sigma = np.full(case["L"], case["sigma"], dtype=np.float32)
        r = oracle.unmix(S, sigma, y[None, :])
        tol = 1e-10 if np.all(x > 0) else 1e-8
        np.testing.assert_allclose(r["x"][0], x, atol=tol, rtol=0)
        assert r["rms"][0] <= 1e-8


def test_closed_form_P1():
    rng = np.random.Generator(np.random.PCG64(5))
    S = rng.uniform(0.2, 0.6, size=(1, 30)).astype(np.float32)
    sigma = np.full(30, 0.01, dtype=np.float32)
    X = rng.uniform(0.0, 1.0, size=(3, 30)).astype(np.float32)
    r = oracle.unmix(S, sigma, X)
    np.testing.assert_array_equal(r["x"], np.ones((3, 1)))
    # one active coordinate: K = [[g, 1],[1, 0]] has K^-1_00 = 0
    np.testing.assert_allclose(r["sx"], 0.0, atol=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_closed_form_P2(seed):
    """x_1 = clamp((c1 - c2 - G12 + G22) / (G11 - 2 G12 + G22), 0, 1)."""
    rng = np.random.Generator(np.random.PCG64(50 + seed))
    L = 40
    S = rng.uniform(0.2, 0.6, size=(2, L)).astype(np.float32)
    sigma = rng.uniform(0.002, 0.02, size=L).astype(np.float32)
    # abundances across [-0.3, 1.3]: both clamped and interior cases
    a = np.linspace(-0.3, 1.3, 9)
    xt = np.stack([a, 1 - a], 1)
    X = (xt @ S.astype(np.float64)).astype(np.float32)
    r = oracle.unmix(S, sigma, X)
    for n in range(len(a)):
        G, c, _ = _pins.qp_terms(S, sigma, X[n])
        x1 = (c[0] - c[1] - G[0, 1] + G[1, 1]) / (G[0, 0] - 2 * G[0, 1] + G[1, 1])
        x1 = min(max(x1, 0.0), 1.0)
        np.testing.assert_allclose(r["x"][n], [x1, 1 - x1], atol=1e-10)


@pytest.mark.parametrize("seed", range(4))
def test_closed_form_interior_scls(seed):
    """All-positive solution: x = G^-1 (c - nu 1), nu = (1'G^-1 c - 1)/(1'G^-1 1)
    (the sum-to-one constrained LS of Sec. 2.2)."""
    rng = np.random.Generator(np.random.PCG64(70 + seed))
    P, L = 5, 60
    S = synth.library(rng, L, P, 0).astype(np.float32)
    sigma = np.full(L, 0.001, dtype=np.float32)
    xt = np.array([0.3, 0.25, 0.2, 0.15, 0.1])
    X = (xt @ S.astype(np.float64) + rng.standard_normal(L) * 0.001).astype(np.float32)[None]
    r = oracle.unmix(S, sigma, X)
    G, c, _ = _pins.qp_terms(S, sigma, X[0])
    Gi_c = np.linalg.solve(G, c)
    Gi_1 = np.linalg.solve(G, np.ones(P))
    nu = (Gi_c.sum() - 1.0) / Gi_1.sum()
    x = Gi_c - nu * Gi_1
    assert np.all(x > 0)
    np.testing.assert_allclose(r["x"][0], x, atol=1e-9)
    np.testing.assert_allclose(r["sx"][0], _pins.support_sigma(G, np.arange(P)), rtol=1e-7)


def test_sigma_scaling_invariance():
    """C -> k^2 C leaves x and the RMS unchanged and scales sigma_x by k."""
    cube = synth.make_cube(synth.OMEGA_262K, n_pix=64)
    base = oracle.unmix(cube.S, cube.sigma, cube.X)
    for k in (0.125, 8.0):
        r = oracle.unmix(cube.S, (cube.sigma * k).astype(np.float32), cube.X)
        np.testing.assert_allclose(r["x"], base["x"], atol=1e-8)
        np.testing.assert_allclose(r["rms"], base["rms"], rtol=1e-7)
        ok = (r["ksup"] == base["ksup"])
        np.testing.assert_allclose(r["sx"][ok], k * base["sx"][ok], rtol=1e-6, atol=1e-12)


def test_permutation_equivariance():
    cube = synth.make_cube(synth.FCLS_1K, n_pix=32)
    perm = np.random.Generator(np.random.PCG64(3)).permutation(cube.P)
    base = oracle.unmix(cube.S, cube.sigma, cube.X)
    r = oracle.unmix(cube.S[perm], cube.sigma, cube.X)
    np.testing.assert_allclose(r["x"], base["x"][:, perm], atol=1e-9)
    np.testing.assert_allclose(r["sx"], base["sx"][:, perm], rtol=1e-6, atol=1e-12)


def test_monte_carlo_uncertainty():
    """Empirical std of x over noise redraws matches sigma_x within 5 %
    (Sec. 2.3: error from the Hessian, read as the estimator's std; the
    paper's F without 1/2 would make it sqrt(2) too small)."""
    rng = np.random.Generator(np.random.PCG64(11))
    P, L = 4, 80
    S = synth.library(rng, L, P, 0).astype(np.float32)
    sigma = rng.uniform(0.002, 0.004, size=L).astype(np.float32)
    xt = np.array([0.35, 0.3, 0.2, 0.15])
    R = 2000
    X = (xt @ S.astype(np.float64) + rng.standard_normal((R, L)) * sigma).astype(np.float32)
    r = oracle.unmix(S, sigma, X)
    assert np.all(r["ksup"] == P), "support not stable: choose a smaller noise"
    emp = r["x"].std(axis=0, ddof=1)
    pred = r["sx"].mean(axis=0)
    np.testing.assert_allclose(emp, pred, rtol=0.05)
    assert np.all(np.abs(r["x"].mean(axis=0) - xt) < 4 * pred / np.sqrt(R) + 1e-12)


def test_rms_definition_and_noise_level():
    """RMS = |y - S^T x| / sqrt(L) (unwhitened) and ~ the noise level on
    exact-model data (Sec. 3.1: RMS compatible with the noise)."""
    cube = synth.make_cube(synth.FCLS_1K, n_pix=300)
    r = oracle.unmix(cube.S, cube.sigma, cube.X)
    fit = r["x"] @ cube.S.astype(np.float64)
    ref = np.sqrt(np.mean((cube.X.astype(np.float64) - fit) ** 2, axis=1))
    np.testing.assert_allclose(r["rms"], ref, rtol=1e-10)
    noise = float(np.sqrt(np.mean(cube.sigma.astype(np.float64) ** 2)))
    assert abs(r["rms"].mean() / noise - 1.0) < 0.05


def test_against_augmented_nnls():
    """FCLS as NNLS with a heavily weighted sum-to-one row (Heinz-Chang);
    its error is O(1/delta^2), independent of the interior-point code."""
    nnls = pytest.importorskip("scipy.optimize").nnls
    cube = synth.make_cube(synth.OMEGA_262K, n_pix=40)
    r = oracle.unmix(cube.S, cube.sigma, cube.X)
    S = cube.S.astype(np.float64)
    w = 1.0 / cube.sigma.astype(np.float64)
    Aw = (S * w).T
    delta = 1e4 * np.sqrt(np.max(np.sum(Aw * Aw, axis=0)))
    Aaug = np.vstack([Aw, delta * np.ones((1, cube.P))])
    for n in range(cube.N):
        yaug = np.concatenate([cube.X[n].astype(np.float64) * w, [delta]])
        xn, _ = nnls(Aaug, yaug, maxiter=50 * cube.P)
        np.testing.assert_allclose(r["x"][n], xn, atol=2e-6)


@pytest.mark.parametrize("P,L,seed", [(36, 184, 1036), (48, 240, 1048)])
def test_large_supports_certified(P, L, seed):
    """Every library column in play (kmax = P) and little noise, the inputs
    of the device's large-support parity case: a quarter to a half of the
    solutions have more than 24 coordinates on their support.  Feasibility,
    a Frank-Wolfe gap ~ 0, the KKT conditions and the augmented NNLS (which
    shares nothing with the interior point) fix the oracle's x there."""
    nnls = pytest.importorskip("scipy.optimize").nnls
    cube = synth.random_instance(seed, 700, L, P, kmax=P, sigma_const=5e-4)
    rows = np.arange(0, cube.N, 7)
    r = oracle.unmix(cube.S, cube.sigma, cube.X[rows])
    assert np.all(r["iters"] >= 0)
    assert np.mean(np.asarray(r["ksup"]) > 24) > 0.2
    G, B = _pins.whiten(cube.S, cube.sigma)
    scale = np.max(np.diag(G))
    w = 1.0 / cube.sigma.astype(np.float64)
    Aw = (cube.S.astype(np.float64) * w).T
    delta = 1e4 * np.sqrt(np.max(np.sum(Aw * Aw, axis=0)))
    Aaug = np.vstack([Aw, delta * np.ones((1, cube.P))])
    for k, n in enumerate(rows):
        x = r["x"][k]
        y = cube.X[n].astype(np.float64)
        c = B @ y
        assert abs(x.sum() - 1.0) <= 1e-12 and x.min() >= 0.0
        assert _pins.fw_gap(G, c, x) <= 1e-9 * scale
        stat, dual = _pins.kkt_violation(G, c, x, support_tol=1e-9)
        assert stat <= 1e-6 * scale and dual <= 1e-6 * scale
        xn, _ = nnls(Aaug, np.concatenate([y * w, [delta]]), maxiter=50 * cube.P)
        np.testing.assert_allclose(x, xn, atol=2e-6)


def test_non_unique_library_detected():
    """The paper's +-cos/+-sin extras (Appendix, ids 37-44) sum to zero in
    pairs; two such pairs give a null direction d of S^T with 1^T d = 0, so
    rank [S^T; 1^T] < P and the minimiser is not unique.  One pair alone
    (1^T d = 2) or the four level/slope extras keep it unique."""
    L = 64
    lam = synth.wavelengths(L)
    u = (lam - lam[0]) / (lam[-1] - lam[0])
    c, s = np.cos(np.pi * u / 2), np.sin(np.pi * u / 2)
    base = [np.ones(L), 0.3 + 0.1 * u]
    assert not synth.check_unique(np.stack(base + [c, -c, s, -s]))
    assert synth.check_unique(np.stack(base + [c, -c]))
    assert synth.check_unique(synth.extra_spectra(L))


# ------------------------------------------------- full noise covariance
def test_cov_diagonal_reduces_to_sigma():
    """C = diag(sigma^2): the full-covariance unmixing is the per-band one."""
    cube = synth.make_cube(synth.OMEGA_262K, n_pix=40)
    Ci = np.diag(1.0 / cube.sigma.astype(np.float64) ** 2)
    a = oracle.unmix_cov(cube.S, Ci, cube.X)
    b = oracle.unmix(cube.S, cube.sigma, cube.X)
    np.testing.assert_allclose(a["x"], b["x"], atol=1e-8)
    np.testing.assert_allclose(a["sx"], b["sx"], rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(a["rms"], b["rms"], rtol=1e-10)


def test_cov_equals_explicit_whitening():
    """With C^-1 = L L^T, whitening the data and the library by L and
    solving with unit noise gives the same x and sigma_x (eq.
    RenormalizedProblem), computed here through an independent path:
    scipy's NNLS on the whitened system with a heavily weighted sum row."""
    from scipy.optimize import nnls
    cube, C, Ci = synth.make_cube_cov(synth.FCLS_1K, 0.6, n_pix=12)
    r = oracle.unmix_cov(cube.S, Ci, cube.X)
    Lc = np.linalg.cholesky(Ci)
    A = cube.S.astype(np.float64) @ Lc          # P x L, whitened library
    w = 1e4
    for n in range(cube.N):
        yw = cube.X[n].astype(np.float64) @ Lc
        M = np.vstack([A.T, w * np.ones((1, A.shape[0]))])
        b = np.concatenate([yw, [w]])
        x, _ = nnls(M, b, maxiter=5000)
        assert np.abs(x / x.sum() - r["x"][n]).max() < 2e-5


def test_cov_scale_invariance_and_kkt():
    """x does not change when C is scaled; sigma_x scales with sqrt(k);
    the KKT conditions of the whitened problem hold."""
    cube, C, Ci = synth.make_cube_cov(synth.OMEGA_262K, 0.5, n_pix=20)
    a = oracle.unmix_cov(cube.S, Ci, cube.X)
    b = oracle.unmix_cov(cube.S, Ci / 4.0, cube.X)
    np.testing.assert_allclose(a["x"], b["x"], atol=1e-8)
    ok = np.abs(a["sx"] * 2.0 - b["sx"]).max(axis=1) < 1e-6
    assert ok.mean() > 0.9
    S = cube.S.astype(np.float64)
    G = S @ Ci @ S.T
    scale = np.trace(G) / cube.P
    for n in range(cube.N):
        c = S @ Ci @ cube.X[n].astype(np.float64)
        assert _pins.fw_gap(G, c, a["x"][n]) <= 1e-9 * scale
        stat, dual = _pins.kkt_violation(G, c, a["x"][n], support_tol=1e-9)
        assert stat <= 1e-6 * scale and dual <= 1e-6 * scale


def test_cov_monte_carlo_sigma():
    """sigma_x under correlated noise (AR(1), rho = 0.7): the empirical std
    of x over noise redraws matches the reported uncertainty within 5 % on
    a problem whose support is stable."""
    rng = np.random.Generator(np.random.PCG64(31))
    P, L = 4, 80
    S = synth.library(rng, L, P, 0).astype(np.float32)
    sigma = rng.uniform(0.002, 0.004, size=L)
    C = synth.ar1_covariance(sigma, 0.7)
    Ci = np.linalg.inv(C)
    Ci = 0.5 * (Ci + Ci.T)
    xt = np.array([0.35, 0.3, 0.2, 0.15])
    R = 2000
    E = rng.standard_normal((R, L)) @ np.linalg.cholesky(C).T
    X = (xt @ S.astype(np.float64) + E).astype(np.float32)
    r = oracle.unmix_cov(S, Ci, X)
    assert np.all(r["x"] > 0.0), "support not stable: choose a smaller noise"
    emp = r["x"].std(axis=0, ddof=1)
    pred = r["sx"].mean(axis=0)
    np.testing.assert_allclose(emp, pred, rtol=0.05)


# ------------------------------------------- slo and pos constraint sets
def _full_rank_instance(seed, N, L, P):
    """Minerals only (no level/slope extras): rank S = P, so that the slo
    and pos minimisers are unique."""
    cube = synth.random_instance(seed, N, L, P, n_extras=0)
    assert np.linalg.matrix_rank(cube.S.astype(np.float64)) == P
    return cube


def test_pos_matches_scipy_nnls():
    """pos is non-negative least squares on the whitened data (scipy)."""
    from scipy.optimize import nnls
    cube = _full_rank_instance(61, 60, 50, 8)
    r = oracle.unmix_constraint(cube.S, cube.sigma, cube.X, "pos")
    assert np.all(r["iters"] > 0)
    w = 1.0 / cube.sigma.astype(np.float64)
    A = (cube.S.astype(np.float64) * w).T
    for n in range(cube.N):
        x, _ = nnls(A, cube.X[n].astype(np.float64) * w, maxiter=5000)
        assert np.abs(x - r["x"][n]).max() <= 1e-6 * max(1.0, x.max())


def test_slo_is_pos_or_sto():
    """slo equals pos where sum x_pos <= 1 and the sum-to-one minimiser
    where sum x_pos > 1 (the inequality is then active); both cases occur."""
    cube = _full_rank_instance(62, 80, 50, 8)
    X = cube.X.astype(np.float64)
    X[::2] *= 1.3                                   # brighter pixels: sum > 1
    X = X.astype(np.float32)
    slo = oracle.unmix_constraint(cube.S, cube.sigma, X, "slo")
    pos = oracle.unmix_constraint(cube.S, cube.sigma, X, "pos")
    sto = oracle.unmix(cube.S, cube.sigma, X)
    tot = pos["x"].sum(1)
    below, above = tot < 1 - 1e-6, tot > 1 + 1e-6
    assert below.sum() > 5 and above.sum() > 5
    np.testing.assert_allclose(slo["x"][below], pos["x"][below], atol=1e-7)
    np.testing.assert_allclose(slo["x"][above], sto["x"][above], atol=1e-7)
    assert np.all(slo["x"].sum(1) <= 1 + 1e-9)
    # uncertainties: the sum is free where the inequality is inactive (pos),
    # bordered where it is active (sto)
    np.testing.assert_allclose(slo["sx"][below], pos["sx"][below], rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(slo["sx"][above], sto["sx"][above], rtol=1e-5, atol=1e-9)


def test_slo_brute_force_supports():
    """Tiny problems: every support with the sum constraint active or not,
    the feasible candidates' best objective equals the oracle's."""
    import itertools
    cube = _full_rank_instance(63, 12, 30, 5)
    X = (cube.X.astype(np.float64) * np.linspace(0.7, 1.4, cube.N)[:, None]).astype(np.float32)
    r = oracle.unmix_constraint(cube.S, cube.sigma, X, "slo")
    G, B = _pins.whiten(cube.S, cube.sigma)
    P = cube.P
    for n in range(cube.N):
        c = B @ X[n].astype(np.float64)
        best, xb = np.inf, None
        for k in range(1, P + 1):
            for S_ in itertools.combinations(range(P), k):
                idx = list(S_)
                Gs, cs = G[np.ix_(idx, idx)], c[idx]
                cands = [np.linalg.solve(Gs, cs)]
                K = np.block([[Gs, np.ones((k, 1))], [np.ones((1, k)), np.zeros((1, 1))]])
                cands.append(np.linalg.solve(K, np.concatenate([cs, [1.0]]))[:k])
                for xs in cands:
                    if xs.min() < -1e-12 or xs.sum() > 1 + 1e-12:
                        continue
                    x = np.zeros(P); x[idx] = xs
                    f = 0.5 * x @ G @ x - c @ x
                    if f < best:
                        best, xb = f, x
        assert np.abs(r["x"][n] - xb).max() <= 1e-7


def test_pos_kkt_and_uncertainty():
    """pos: gradient ~0 on the support, >= 0 off it; the uncertainty is
    sqrt(diag(G_SS^-1)) on the support (no sum constraint), 0 off it."""
    cube = _full_rank_instance(64, 30, 60, 10)
    r = oracle.unmix_constraint(cube.S, cube.sigma, cube.X, "pos")
    G, B = _pins.whiten(cube.S, cube.sigma)
    scale = np.max(np.diag(G))
    for n in range(cube.N):
        x = r["x"][n]
        g = G @ x - B @ cube.X[n].astype(np.float64)
        S_ = x > 1e-9
        assert np.abs(g[S_]).max() <= 1e-6 * scale
        if (~S_).any():
            assert g[~S_].min() >= -1e-6 * scale
        idx = np.flatnonzero(S_)
        ratio = r["lam"][n] / np.maximum(x, 1e-300) / np.diag(G)
        if np.any((ratio > 1e-3) & (ratio < 1e3)):
            continue                                 # no strict complementarity
        sx = np.sqrt(np.diag(np.linalg.inv(G[np.ix_(idx, idx)])))
        np.testing.assert_allclose(r["sx"][n][idx], sx, rtol=1e-6)
        assert np.all(r["sx"][n][~S_] == 0.0)


def test_pos_brute_force_supports():
    """Tiny problems: the pos minimiser is the best feasible unconstrained
    least-squares solution over all supports (no sum constraint at all,
    so sums well above 1 occur)."""
    import itertools
    cube = _full_rank_instance(65, 12, 30, 5)
    X = (cube.X.astype(np.float64) * np.linspace(0.5, 3.0, cube.N)[:, None]).astype(np.float32)
    r = oracle.unmix_constraint(cube.S, cube.sigma, X, "pos")
    G, B = _pins.whiten(cube.S, cube.sigma)
    P = cube.P
    assert r["x"].sum(1).max() > 2.0
    for n in range(cube.N):
        c = B @ X[n].astype(np.float64)
        best, xb = 0.0, np.zeros(P)            # the empty support: x = 0, f = 0
        for k in range(1, P + 1):
            for S_ in itertools.combinations(range(P), k):
                idx = list(S_)
                xs = np.linalg.solve(G[np.ix_(idx, idx)], c[idx])
                if xs.min() < -1e-12:
                    continue
                x = np.zeros(P); x[idx] = xs
                f = 0.5 * x @ G @ x - c @ x
                if f < best:
                    best, xb = f, x
        assert np.abs(r["x"][n] - xb).max() <= 1e-7 * max(1.0, xb.max())


def test_slo_kkt_certificate():
    """slo: gradient + omega vanishes on the support and is >= 0 off it;
    omega >= 0, slack w = 1 - sum x >= 0 and w omega ~ 0 (one of the two is
    negligible on every pixel)."""
    cube = _full_rank_instance(66, 60, 50, 8)
    X = (cube.X.astype(np.float64) * np.linspace(0.6, 1.5, cube.N)[:, None]).astype(np.float32)
    r = oracle.unmix_constraint(cube.S, cube.sigma, X, "slo")
    assert np.all(r["iters"] > 0)
    G, B = _pins.whiten(cube.S, cube.sigma)
    scale = np.max(np.diag(G))
    np.testing.assert_allclose(r["slack"], 1.0 - r["x"].sum(1), atol=1e-12)
    assert np.all(r["slack"] >= -1e-14) and np.all(r["omega"] >= 0.0)
    assert np.all(np.minimum(r["slack"], r["omega"] / scale) <= 1e-9)
    for n in range(cube.N):
        x = r["x"][n]
        g = G @ x - B @ X[n].astype(np.float64) + r["omega"][n]
        S_ = x > 1e-9
        assert np.abs(g[S_]).max() <= 1e-6 * scale
        if (~S_).any():
            assert g[~S_].min() >= -1e-6 * scale


# Pixels of the seeded full-size workloads on which the interior point, with
# separate primal and dual step lengths and no centring fallback, stalled
# (the dual residual stuck, or a two-iteration cycle between near-dependent
# spectra with mu bouncing between two values).
HARD_PIXELS = {"omega_262k_L184_P36": [107698, 118302, 126310, 135370, 161210, 211715,
                                       218946, 260039],
               "crism_307k_L240_P48": [204239]}


@pytest.mark.parametrize("name", sorted(HARD_PIXELS))
def test_converges_on_pixels_that_stalled(name):
    """Every solve converges (stop test met, not the cap) and its result is
    the minimiser: the Frank-Wolfe gap (an upper bound on f(x) - f*) is at
    the rounding level of the problem."""
    spec = [w for w in synth.WORKLOADS if w.name == name][0]
    idx = HARD_PIXELS[name]
    cube = synth.make_cube(spec, n_pix=max(idx) + 1)
    r = oracle.unmix(cube.S, cube.sigma, cube.X[idx])
    assert np.all(r["iters"] > 0) and np.all(r["status"] == 0)
    G, B = _pins.whiten(cube.S, cube.sigma)
    scale = np.trace(G) / G.shape[0]
    for k, n in enumerate(idx):
        c = B @ cube.X[n].astype(np.float64)
        assert _pins.fw_gap(G, c, r["x"][k]) <= 1e-9 * scale

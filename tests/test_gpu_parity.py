"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (written here, derived from the problem):
  * abundances: max |x_gpu - x_oracle| <= 1e-4 per abundance;
  * objective: f(x_gpu) - f(x*) <= 1e-6 |f(x*)| with f evaluated in fp64;
  * uncertainties: max |sx_gpu - sx_oracle| <= 1e-4 on pixels whose support
    is unambiguous (every coordinate has lambda_i / (x_i G_ii) outside
    [1e-3, 1e3] at the oracle's solution; without strict complementarity
    the support, hence the covariance, is not defined by the data);
  * rms: relative 1e-4 (float32 evaluation of an O(1e-2) residual of O(1)
    terms loses ~1e-5, and x differs by <= 1e-4);
  * sum-to-one exact to 1e-5 in float32, x >= 0.
Small configurations are compared element by element; the full-size
workloads run in the launch configuration the benchmark uses and are
compared on a seeded sample of pixels the oracle recomputes one by one.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import _pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

X_TOL = 1e-4
SX_TOL = 1e-4
RMS_RTOL = 1e-4


@pytest.fixture(scope="module")
def pkg():
    import paper_1402_2518_gb300 as p
    p.load()
    return p


def run_gpu(pkg, S, sigma, X, **kw):
    dev = torch.device("cuda:0")
    um = pkg.Unmixer(torch.from_numpy(np.ascontiguousarray(S)).to(dev), **kw)
    x, sx, rms, it = um(torch.from_numpy(np.ascontiguousarray(X)).to(dev),
                        torch.from_numpy(np.ascontiguousarray(sigma)).to(dev))
    st, nbad = um.wait()
    out = dict(x=x.cpu().numpy().astype(np.float64), sx=sx.cpu().numpy().astype(np.float64),
               rms=rms.cpu().numpy().astype(np.float64), iters=it.cpu().numpy(),
               status=st, n_notconv=nbad)
    um.close()
    return out


def unambiguous(ref, S, sigma):
    """Pixels whose support is resolved by the data (reading of the
    uncertainty definition, Sec. 2.3: the covariance is taken on the support
    of the solution, which strict complementarity must fix).  A coordinate
    is ambiguous when lambda_i / (x_i G_ii) lies in [1e-3, 1e3], or when
    its margin, in the scaled units of the solver (G / s, s = trace(G) / P),
    is below 1e-8: for an inactive coordinate the margin is its multiplier
    lambda_i, for an active one the multiplier that dropping it would leave,
    x_i / sigma_i^2 (the diagonal of the bordered inverse is sigma^2).  A
    margin below 1e-8 is within 10x of the exactness stage's acceptance
    tolerance and below the ~6e-8 relative rounding of float32 input data,
    so either support is consistent with the data."""
    G, _ = _pins.whiten(S, sigma)
    s = np.trace(G) / G.shape[0]
    x, lam = ref["x"], ref["lam"]
    ratio = lam / np.maximum(x, 1e-300) / np.diag(G)[None, :]
    active = ratio < 1e-3
    with np.errstate(divide="ignore"):
        margin = np.where(active, x / np.maximum(ref["sx"], 1e-300) ** 2, lam) / s
    return ~np.any((ratio > 1e-3) & (ratio < 1e3), axis=1) & np.all(margin >= 1e-8, axis=1)


def check(gpu, ref, S, sigma, X, rows=None):
    rows = np.arange(X.shape[0]) if rows is None else rows
    xg, sg, rg = gpu["x"][rows], gpu["sx"][rows], gpu["rms"][rows]
    assert gpu["n_notconv"] == 0 and np.all(gpu["iters"][rows] >= 0)
    assert np.all(xg >= 0.0)
    np.testing.assert_allclose(xg.sum(axis=1), 1.0, atol=1e-5)
    err = np.abs(xg - ref["x"]).max()
    assert err <= X_TOL, f"max |x_gpu - x_oracle| = {err:.3e}"
    G, B = _pins.whiten(S, sigma)
    for k, n in enumerate(rows):
        y = X[n].astype(np.float64)
        c = B @ y
        s = float(np.sum(y * y / sigma.astype(np.float64) ** 2))
        f_or = _pins.objective(G, c, s, ref["x"][k])
        f_gp = _pins.objective(G, c, s, xg[k] / xg[k].sum())
        assert f_gp - f_or <= 1e-6 * abs(f_or) + 1e-9, (n, f_gp, f_or)
    ok = unambiguous(ref, S, sigma)
    assert ok.mean() > 0.8
    serr = np.abs(sg[ok] - ref["sx"][ok]).max()
    assert serr <= SX_TOL, f"max |sx_gpu - sx_oracle| = {serr:.3e}"
    np.testing.assert_allclose(rg, ref["rms"], rtol=RMS_RTOL)
    return err, serr


@pytest.mark.parametrize("spec", synth.WORKLOADS, ids=lambda s: s.name)
def test_small_prefix_elementwise(pkg, spec):
    """Every pixel of a 2000-pixel prefix (several groups and blocks, a
    ragged tail of the last block)."""
    cube = synth.make_cube(spec, n_pix=2000 if spec.n_pix > 2000 else None)
    ref = oracle.unmix(cube.S, cube.sigma, cube.X)
    gpu = run_gpu(pkg, cube.S, cube.sigma, cube.X)
    check(gpu, ref, cube.S, cube.sigma, cube.X)


@pytest.mark.parametrize("spec", synth.WORKLOADS[1:], ids=lambda s: s.name)
def test_full_size_sampled(pkg, spec):
    """The full cube in the benchmark's launch configuration; 1500 seeded
    pixels recomputed by the oracle."""
    cube = synth.make_cube(spec)
    gpu = run_gpu(pkg, cube.S, cube.sigma, cube.X)
    rng = np.random.Generator(np.random.PCG64(99))
    rows = np.sort(rng.choice(cube.N, size=1500, replace=False))
    rows[-1] = cube.N - 1                       # include the very last pixel
    ref = oracle.unmix(cube.S, cube.sigma, cube.X[rows])
    check(gpu, ref, cube.S, cube.sigma, cube.X, rows)
    # properties that hold at every pixel
    assert np.all(gpu["iters"] > 0)
    assert np.all(gpu["x"] >= 0)
    np.testing.assert_allclose(gpu["x"].sum(1), 1.0, atol=1e-5)


@pytest.mark.parametrize("seed", range(8))
def test_random_small_libraries(pkg, seed):
    """Odd P (padded rows in every kernel bucket), extras, ragged N."""
    rng = np.random.Generator(np.random.PCG64(500 + seed))
    P = int(rng.choice([2, 3, 5, 7, 9, 13, 17, 23, 31, 37, 41, 47]))
    L = int(rng.integers(P + 3, 3 * P + 40))
    extras = 4 if P >= 8 and seed % 2 == 0 else 0
    N = int(rng.integers(1, 700))
    cube = synth.random_instance(800 + seed, N, L, P, n_extras=extras)
    ref = oracle.unmix(cube.S, cube.sigma, cube.X)
    gpu = run_gpu(pkg, cube.S, cube.sigma, cube.X)
    check(gpu, ref, cube.S, cube.sigma, cube.X)


@pytest.mark.parametrize("P", [49, 57, 64])
def test_large_libraries(pkg, P):
    """The P <= 64 size bucket (16 lanes per pixel, padded rows for P < 64)."""
    cube = synth.random_instance(900 + P, 300, P + 40, P, n_extras=4, kmax=5)
    ref = oracle.unmix(cube.S, cube.sigma, cube.X)
    gpu = run_gpu(pkg, cube.S, cube.sigma, cube.X)
    check(gpu, ref, cube.S, cube.sigma, cube.X)


@pytest.mark.parametrize("P,L,seed", [(36, 184, 1036), (48, 240, 1048)])
def test_large_supports(pkg, P, L, seed):
    """Every library column in play (kmax = P) and little noise: about a
    third (P = 36) to two thirds (P = 48) of the solutions have more than 24
    coordinates on their support, so the crossover's lane groups hand those
    pixels from the launch that holds supports of at most 24 coordinates to
    the one sized by P."""
    cube = synth.random_instance(seed, 700, L, P, kmax=P, sigma_const=5e-4)
    ref = oracle.unmix(cube.S, cube.sigma, cube.X)
    assert np.mean(np.asarray(ref["ksup"]) > 24) > 0.25
    gpu = run_gpu(pkg, cube.S, cube.sigma, cube.X)
    check(gpu, ref, cube.S, cube.sigma, cube.X)


def test_P1_and_N1(pkg):
    rng = np.random.Generator(np.random.PCG64(7))
    S = rng.uniform(0.2, 0.6, (1, 20)).astype(np.float32)
    sig = np.full(20, 0.01, np.float32)
    X = rng.uniform(0.1, 0.7, (5, 20)).astype(np.float32)
    gpu = run_gpu(pkg, S, sig, X)
    np.testing.assert_array_equal(gpu["x"], 1.0)
    np.testing.assert_allclose(gpu["sx"], 0.0, atol=1e-6)
    cube = synth.make_cube(synth.FCLS_1K, n_pix=1)
    ref = oracle.unmix(cube.S, cube.sigma, cube.X)
    check(run_gpu(pkg, cube.S, cube.sigma, cube.X), ref, cube.S, cube.sigma, cube.X)


def test_exact_mixtures(pkg):
    """Noise-free dyadic mixtures (tests/golden): x recovered to 1e-5."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "dyadic_mixtures.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        S = (np.array(case["S_num"], np.float64) / case["S_den"]).astype(np.float32)
        x = np.array(case["x"])
        y = (x @ S.astype(np.float64)).astype(np.float32)[None]
        sig = np.full(case["L"], case["sigma"], np.float32)
        gpu = run_gpu(pkg, S, sig, y)
        np.testing.assert_allclose(gpu["x"][0], x, atol=1e-5)


def test_host_pointers_match_device(pkg):
    """The host-buffer path (copies inside the call) gives the same bits."""
    cube = synth.make_cube(synth.OMEGA_262K, n_pix=3000)
    gpu = run_gpu(pkg, cube.S, cube.sigma, cube.X)
    h = pkg.linmin_create(cube.S, cube.L, cube.P)
    x = np.empty((cube.N, cube.P), np.float32); sx = np.empty_like(x)
    rms = np.empty(cube.N, np.float32); it = np.empty(cube.N, np.int32)
    st = pkg.linmin_unmix(h, cube.X, cube.N, cube.sigma, x, sx, rms, it)
    pkg.linmin_destroy(h)
    assert st == 0
    np.testing.assert_array_equal(x, gpu["x"].astype(np.float32))
    np.testing.assert_array_equal(sx, gpu["sx"].astype(np.float32))
    np.testing.assert_array_equal(rms, gpu["rms"].astype(np.float32))
    np.testing.assert_array_equal(it, gpu["iters"])


def test_same_result_alone_and_in_a_batch(pkg):
    """Per-pixel work does not depend on placement: a pixel gives the same
    bits alone, in a small batch and in a large one."""
    cube = synth.make_cube(synth.OMEGA_262K, n_pix=5000)
    full = run_gpu(pkg, cube.S, cube.sigma, cube.X)
    for lo, hi in [(0, 1), (1234, 1300), (4999, 5000)]:
        part = run_gpu(pkg, cube.S, cube.sigma, cube.X[lo:hi])
        np.testing.assert_array_equal(part["x"], full["x"][lo:hi])
        np.testing.assert_array_equal(part["sx"], full["sx"][lo:hi])


def test_sigma_scaling_invariance(pkg):
    cube = synth.make_cube(synth.OMEGA_262K, n_pix=1000)
    a = run_gpu(pkg, cube.S, cube.sigma, cube.X)
    b = run_gpu(pkg, cube.S, (cube.sigma * 8).astype(np.float32), cube.X)
    assert np.abs(a["x"] - b["x"]).max() <= 2e-5
    ok = np.abs(a["sx"] * 8 - b["sx"]).max(axis=1) < 1e-3
    assert ok.mean() > 0.99


def test_not_converged_reported(pkg):
    """With a 1-iteration cap the crossover still finishes many pixels
    exactly; the rest hit the cap on the retry path.  Negative iteration
    counts, the reported count and the status agree, and every pixel that
    is reported converged is correct."""
    cube = synth.make_cube(synth.OMEGA_262K, n_pix=300)
    gpu = run_gpu(pkg, cube.S, cube.sigma, cube.X, max_iter=1)
    bad = gpu["iters"] < 0
    assert gpu["n_notconv"] == int(bad.sum())
    assert gpu["status"] == (6 if bad.any() else 0)
    assert bad.any(), "a 1-iteration cap should leave some pixels unfinished"
    ref = oracle.unmix(cube.S, cube.sigma, cube.X)
    good = ~bad
    assert np.abs(gpu["x"][good] - ref["x"][good]).max() <= X_TOL


def test_invalid_sigma_and_empty(pkg):
    cube = synth.make_cube(synth.FCLS_1K, n_pix=10)
    h = pkg.linmin_create(cube.S, cube.L, cube.P)
    bad = cube.sigma.copy(); bad[3] = 0.0
    x = np.empty((10, cube.P), np.float32)
    assert pkg.linmin_unmix(h, cube.X, 10, bad, x, check=False) == 1
    assert pkg.linmin_unmix(h, cube.X, 0, cube.sigma, x) == 0
    # device sigma: checked on the device, reported by linmin_wait
    dev = torch.device("cuda:0")
    Xd = torch.from_numpy(cube.X).to(dev)
    bd = torch.from_numpy(bad).to(dev)
    xd = torch.empty((10, cube.P), device=dev)
    pkg.linmin_unmix(h, Xd, 10, bd, xd, check=False)
    st, _ = pkg.linmin_wait(h)
    assert st == 1
    pkg.linmin_destroy(h)

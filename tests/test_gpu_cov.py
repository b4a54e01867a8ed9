"""Unmixing under a full noise covariance (linmin_unmix_cov) against the
FP64 oracle (oracle.unmix_cov): band-correlated AR(1) noise, the same bars
as the per-band path (x 1e-4, objective 1e-6 relative, uncertainties 1e-4
on pixels with an unambiguous support, RMS 1e-4 relative)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def pkg():
    import paper_1402_2518_gb300 as p
    p.load()
    return p


def run_cov(pkg, S, Ci, X, device=True):
    dev = torch.device(DEV)
    N, P = X.shape[0], S.shape[0]
    h = pkg.linmin_create(torch.from_numpy(S).to(dev), S.shape[1], P)
    Xd = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    Cd = torch.from_numpy(np.ascontiguousarray(Ci)).to(dev) if device else np.ascontiguousarray(Ci)
    x = torch.empty((N, P), device=dev); sx = torch.empty((N, P), device=dev)
    rms = torch.empty((N,), device=dev); it = torch.empty((N,), dtype=torch.int32, device=dev)
    pkg.linmin_unmix_cov(h, Xd, N, Cd, x, sx, rms, it)
    st, nbad = pkg.linmin_wait(h)
    launches = pkg.linmin_last_launches(h)
    pkg.linmin_destroy(h)
    return st, nbad, launches, [t.cpu().numpy() for t in (x, sx, rms, it)]


def check(S, Ci, X, got, ref, rows):
    x, sx, rms, it = (a[rows] for a in got)
    assert np.all(it > 0) and np.all(x >= 0)
    np.testing.assert_allclose(x.sum(1), 1.0, atol=1e-5)
    assert np.abs(x - ref["x"]).max() <= 1e-4
    G = ref["G"]
    S64 = S.astype(np.float64)
    for k, n in enumerate(rows):
        c = S64 @ Ci @ X[n].astype(np.float64)
        f = lambda v: 0.5 * v @ G @ v - c @ v
        xg = x[k].astype(np.float64); xg /= xg.sum()
        assert f(xg) - f(ref["x"][k]) <= 1e-6 * abs(f(ref["x"][k])) + 1e-9
    ratio = ref["lam"] / np.maximum(ref["x"], 1e-300) / np.diag(G)[None, :]
    ok = ~np.any((ratio > 1e-3) & (ratio < 1e3), axis=1)
    assert ok.mean() > 0.8
    assert np.abs(sx[ok] - ref["sx"][ok]).max() <= 1e-4
    np.testing.assert_allclose(rms, ref["rms"], rtol=1e-4)


@pytest.mark.parametrize("spec,rho", [(synth.FCLS_1K, 0.6), (synth.OMEGA_262K, 0.5),
                                      (synth.CRISM_307K, 0.3)], ids=["fcls1k", "omega", "crism"])
def test_cov_prefix_elementwise(pkg, spec, rho):
    cube, C, Ci = synth.make_cube_cov(spec, rho, n_pix=1200)
    st, nbad, launches, got = run_cov(pkg, cube.S, Ci, cube.X)
    assert st == 0 and nbad == 0
    assert launches == 4 + 4 + 1 + 9 + 2 + 3 + 1         # cov prep 4, tensor-core projection 4
    ref = oracle.unmix_cov(cube.S, Ci, cube.X)
    check(cube.S, Ci, cube.X, got, ref, np.arange(cube.N))


def test_cov_full_size_sampled(pkg):
    """The 262,144-pixel cube with AR(1) noise; 600 seeded pixels."""
    cube, C, Ci = synth.make_cube_cov(synth.OMEGA_262K, 0.5)
    st, nbad, _, got = run_cov(pkg, cube.S, Ci, cube.X)
    assert st == 0 and nbad == 0
    rng = np.random.Generator(np.random.PCG64(5))
    rows = np.sort(rng.choice(cube.N, size=600, replace=False))
    ref = oracle.unmix_cov(cube.S, Ci, cube.X[rows])
    check(cube.S, Ci, cube.X, got, ref, rows)


def test_cov_diagonal_matches_sigma_path(pkg):
    cube = synth.make_cube(synth.OMEGA_262K, n_pix=2000)
    Ci = np.diag(1.0 / cube.sigma.astype(np.float64) ** 2)
    _, _, _, a = run_cov(pkg, cube.S, Ci, cube.X)
    dev = torch.device(DEV)
    um = pkg.Unmixer(torch.from_numpy(cube.S).to(dev))
    x, sx, rms, it = um(torch.from_numpy(cube.X).to(dev), torch.from_numpy(cube.sigma).to(dev))
    um.wait(); um.close()
    assert np.abs(a[0] - x.cpu().numpy()).max() <= 1e-6
    np.testing.assert_allclose(a[2], rms.cpu().numpy(), rtol=1e-5)


def test_cov_host_equals_device_and_invalid(pkg):
    from paper_1402_2518_gb300 import linmin
    cube, C, Ci = synth.make_cube_cov(synth.FCLS_1K, 0.6, n_pix=500)
    _, _, _, a = run_cov(pkg, cube.S, Ci, cube.X, device=True)
    _, _, _, b = run_cov(pkg, cube.S, Ci, cube.X, device=False)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    h = pkg.linmin_create(cube.S, cube.L, cube.P)
    x = np.empty((cube.N, cube.P), np.float32)
    for bad in (-np.eye(cube.L), Ci + np.triu(np.ones_like(Ci), 1) * 1e-3,
                np.where(np.eye(cube.L) > 0, np.nan, Ci)):
        bad = np.ascontiguousarray(bad, dtype=np.float64)
        assert pkg.linmin_unmix_cov(h, cube.X, cube.N, bad, x, check=False) == \
            linmin.LINMIN_ERR_INVALID
    assert pkg.linmin_unmix_cov(h, cube.X, cube.N, None, x, check=False) == \
        linmin.LINMIN_ERR_INVALID
    pkg.linmin_destroy(h)

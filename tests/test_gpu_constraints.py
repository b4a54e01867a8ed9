"""The slo (sum x <= 1) and pos (x >= 0) constraint sets on the device
against the oracle (oracle.unmix_constraint: interior-point methods written
from each set's own definition), with the same bars as the
sum-to-one path: x 1e-4, uncertainties 1e-4 on unambiguous pixels, RMS 1e-4
relative.  Libraries have rank S = P (minerals, or the OMEGA-shaped library
without its decreasing slope)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
NAMES = {"slo": 1, "pos": 2}


@pytest.fixture(scope="module")
def pkg():
    import paper_1402_2518_gb300 as p
    p.load()
    return p


def run(pkg, S, sigma, X, constraint):
    dev = torch.device(DEV)
    um = pkg.Unmixer(torch.from_numpy(np.ascontiguousarray(S)).to(dev),
                     constraint=NAMES[constraint])
    x, sx, rms, it = um(torch.from_numpy(np.ascontiguousarray(X)).to(dev),
                        torch.from_numpy(np.ascontiguousarray(sigma)).to(dev))
    st, nbad = um.wait()
    um.close()
    return st, nbad, [t.cpu().numpy().astype(np.float64) for t in (x, sx, rms)] + [it.cpu().numpy()]


def omega_rank_full(n_pix):
    cube = synth.make_cube(synth.OMEGA_262K, n_pix=n_pix)
    keep = [j for j in range(cube.P) if j != cube.P - 2]       # drop 0.5 (1 - u)
    S = np.ascontiguousarray(cube.S[keep])
    assert np.linalg.matrix_rank(S.astype(np.float64)) == S.shape[0]
    return S, cube.sigma, cube.X


def check(got, ref, S, sigma):
    x, sx, rms, it = got
    assert np.all(it > 0) and np.all(x >= 0)
    assert np.abs(x - ref["x"]).max() <= 1e-4
    w2 = 1.0 / sigma.astype(np.float64) ** 2
    gd = (S.astype(np.float64) ** 2 * w2).sum(1)
    ratio = ref["lam"] / np.maximum(ref["x"], 1e-300) / gd[None, :]
    ok = ~np.any((ratio > 1e-3) & (ratio < 1e3), axis=1)
    assert ok.mean() > 0.7
    assert np.abs(sx[ok] - ref["sx"][ok]).max() <= 1e-4 * max(1.0, np.abs(ref["sx"][ok]).max())
    np.testing.assert_allclose(rms, ref["rms"], rtol=1e-4)


@pytest.mark.parametrize("constraint", ["slo", "pos"])
def test_random_full_rank(pkg, constraint):
    cube = synth.random_instance(3300, 700, 96, 20, n_extras=0)
    X = (cube.X.astype(np.float64) * np.linspace(0.6, 1.5, cube.N)[:, None]).astype(np.float32)
    ref = oracle.unmix_constraint(cube.S, cube.sigma, X, constraint)
    st, nbad, got = run(pkg, cube.S, cube.sigma, X, constraint)
    assert st == 0 and nbad == 0
    check(got, ref, cube.S, cube.sigma)
    if constraint == "slo":
        assert np.all(got[0].sum(1) <= 1 + 1e-5)
        tot = ref["x"].sum(1)
        assert (tot < 1 - 1e-3).sum() > 20 and (tot > 1 - 1e-6).sum() > 20   # both regimes


@pytest.mark.parametrize("constraint", ["slo", "pos"])
def test_omega_shaped(pkg, constraint):
    S, sigma, X = omega_rank_full(1500)
    ref = oracle.unmix_constraint(S, sigma, X, constraint)
    st, nbad, got = run(pkg, S, sigma, X, constraint)
    assert st == 0 and nbad == 0
    check(got, ref, S, sigma)


@pytest.mark.parametrize("constraint", ["slo", "pos"])
def test_omega_full_size_converges(pkg, constraint):
    """Every pixel of the full 262,144-pixel OMEGA-shaped cube converges
    under slo and pos, and a seeded sample of 512 pixels matches the oracle.
    The pos thresholds sit at the float32 floor, where even the summation
    order of the dual residual decides whether a pixel reaches them: this
    catches a change of rounding that leaves pixels at the iteration cap."""
    S, sigma, X = omega_rank_full(None)
    st, nbad, got = run(pkg, S, sigma, X, constraint)
    assert st == 0 and nbad == 0
    rows = np.sort(np.random.default_rng(11).choice(X.shape[0], 512, replace=False))
    ref = oracle.unmix_constraint(S, sigma, X[rows], constraint)
    check([g[rows] for g in got], ref, S, sigma)


def test_rank_and_size_refusals(pkg):
    from paper_1402_2518_gb300 import linmin
    cube = synth.make_cube(synth.OMEGA_262K, n_pix=4)          # flat + slopes: rank S = P - 1
    for c in (1, 2):
        opt = pkg.linmin_default_options()
        opt.constraint = c
        with pytest.raises(linmin.LinminError) as e:
            pkg.linmin_create(cube.S, cube.L, cube.P, opt)
        assert e.value.status == linmin.LINMIN_ERR_RANK
    big = synth.random_instance(3301, 2, 100, 64, n_extras=0)
    opt = pkg.linmin_default_options()
    opt.constraint = 1
    with pytest.raises(linmin.LinminError) as e:
        pkg.linmin_create(big.S, big.L, big.P, opt)
    assert e.value.status == linmin.LINMIN_ERR_UNSUPPORTED


def test_pos_sum_bound_is_flagged(pkg):
    """The device solves pos as slo on M S with M = LINMIN_POS_SCALE, which is
    exact while sum x < M.  A pixel whose pos minimiser has a larger sum is
    reported, not silently clipped: negative iteration count and
    LINMIN_ERR_NOT_CONVERGED; every other pixel still matches the oracle."""
    from paper_1402_2518_gb300 import linmin
    cube = synth.random_instance(3302, 200, 96, 12, n_extras=0)
    X = cube.X.astype(np.float64).copy()
    big = np.arange(0, cube.N, 10)
    X[big] = X[big] * (2.0 * linmin.LINMIN_POS_SCALE)          # sums near 2 M
    X = X.astype(np.float32)
    ref = oracle.unmix_constraint(cube.S, cube.sigma, X, "pos")
    over = ref["x"].sum(1) >= linmin.LINMIN_POS_SCALE
    assert over[big].all() and not over[np.setdiff1d(np.arange(cube.N), big)].any()
    st, nbad, got = run(pkg, cube.S, cube.sigma, X, "pos")
    x, sx, rms, it = got
    assert st == linmin.LINMIN_ERR_NOT_CONVERGED and nbad == over.sum()
    assert np.all(it[over] < 0) and np.all(it[~over] > 0)
    assert np.abs(x[~over] - ref["x"][~over]).max() <= 1e-4

"""Second pass of Sec. 5 on the device through the C ABI against the
oracle (oracle.detection.second_pass), on the same masks: the oracle's own
detections on the surface mixtures of Sec. 3.1, the true minerals, and
random masks over many groups with a ragged pixel count."""
import numpy as np
import pytest

import oracle
import oracle.detection as od
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def pkg():
    import paper_1402_2518_gb300 as p
    p.load()
    return p


def _d(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).to(DEV)


def run(pkg, S, X, sigma, mask, nm):
    N, P = X.shape[0], S.shape[0]
    x = torch.full((max(N, 1), P), np.nan, device=DEV)
    sx = torch.full((max(N, 1), P), np.nan, device=DEV)
    rms = torch.full((max(N, 1),), np.nan, device=DEV)
    it = torch.zeros((max(N, 1),), dtype=torch.int32, device=DEV)
    dummy = torch.zeros((1,), dtype=torch.int64, device=DEV)
    st = pkg.linmin_second_pass(_d(S), S.shape[1], P, nm, _d(X) if N else x, N, _d(sigma),
                                _d(mask) if N else dummy, x, sx, rms, it)
    torch.cuda.synchronize()
    return st, [t[:N].cpu().numpy().astype(np.float64) for t in (x, sx, rms)] + [it[:N].cpu().numpy()]


def check(got, ref, mask, nm, S, sigma):
    x, sx, rms, it = got
    P = x.shape[1]
    assert (it > 0).all()
    assert np.abs(x - ref["x"]).max() <= 1e-4
    bits = ((np.asarray(mask, np.uint64)[:, None] >> np.arange(P, dtype=np.uint64)[None, :])
            & np.uint64(1)).astype(bool)
    off = ~bits & (np.arange(P)[None, :] < nm)
    assert (x[off] == 0).all() and (sx[off] == 0).all()
    np.testing.assert_allclose(rms, ref["rms"], rtol=1e-4)
    # uncertainties on pixels without a coordinate near degeneracy, where
    # the support is ambiguous: x_i and lambda_i both small relative to
    # each other, or a decision margin below the crossover's resolution
    # (1e-9 of s = trace(G)/P in the gradient): a support coordinate whose
    # removal would move the gradient by only x_i / sigma_i^2 (its
    # effective curvature is 1 / sigma_i^2), or an excluded one whose
    # multiplier lambda_i is that small
    w2 = 1.0 / sigma.astype(np.float64) ** 2
    gd = (S.astype(np.float64) ** 2 * w2).sum(1)
    s = gd.mean()
    ratio = ref["lam"] / np.maximum(ref["x"], 1e-300) / gd[None, :]
    sup = ref["sx"] > 0
    amb_in = sup & (ref["x"] / np.maximum(ref["sx"] ** 2, 1e-300) / s < 1e-8)
    amb_out = ~sup & ~off & (ref["lam"] / s < 1e-8)
    ok = ~np.any(((ratio > 1e-3) & (ratio < 1e3)) | amb_in | amb_out, axis=1)
    assert ok.mean() > 0.7
    assert np.abs(sx[ok] - ref["sx"][ok]).max() <= 1e-4 * max(1.0, np.abs(ref["sx"][ok]).max())


def test_second_pass_on_detections(pkg):
    cube, truth = synth.surface_mixtures()
    nm = 32
    first = oracle.unmix(cube.S, cube.sigma, cube.X)
    C = np.maximum(od.thresholds(first["x"], truth, nm), 0).astype(np.float32)
    det = od.detect(first["x"].astype(np.float32), first["sx"].astype(np.float32),
                    first["rms"].astype(np.float32), first["iters"], truth, C,
                    float(2 * cube.sigma.mean()), nm)
    st, got = run(pkg, cube.S, cube.X, cube.sigma, det["mask"], nm)
    ref = od.second_pass(cube.S, cube.sigma, cube.X, det["mask"], nm)
    assert st == 0
    check(got, ref, det["mask"], nm, cube.S, cube.sigma)


def test_second_pass_true_minerals_sharpen(pkg):
    """With the minerals that are really there, the second pass brings the
    abundances closer to the truth than the first (the claim of Sec. 5)."""
    cube, truth = synth.surface_mixtures()
    nm = 32
    st, got = run(pkg, cube.S, cube.X, cube.sigma, truth, nm)
    ref = od.second_pass(cube.S, cube.sigma, cube.X, truth, nm)
    assert st == 0
    check(got, ref, truth, nm, cube.S, cube.sigma)
    first = oracle.unmix(cube.S, cube.sigma, cube.X)
    pres = cube.A_true[:, :nm] > 0
    e1 = np.abs(first["x"][:, :nm][pres] - cube.A_true[:, :nm][pres]).mean()
    e2 = np.abs(got[0][:, :nm][pres] - cube.A_true[:, :nm][pres]).mean()
    print(f"mean |x - x_true| of present minerals: first pass {e1:.4f}, second pass {e2:.4f}")
    assert e2 < e1


def test_second_pass_random_masks(pkg):
    cube = synth.random_instance(61, 3001, 128, 20, n_extras=4)
    nm = 16
    rng = np.random.Generator(np.random.PCG64(62))
    masks = rng.integers(0, 1 << 5, cube.N).astype(np.uint64) << np.uint64(3)   # 32 groups
    masks[rng.random(cube.N) < 0.1] = 0                                      # extras only
    masks[:7] = np.uint64((1 << nm) - 1) | np.uint64(1 << 40)                # high bits ignored
    st, got = run(pkg, cube.S, cube.X, cube.sigma, masks, nm)
    ref = od.second_pass(cube.S, cube.sigma, cube.X, masks, nm)
    assert st == 0
    check(got, ref, masks, nm, cube.S, cube.sigma)


def test_second_pass_empty(pkg):
    cube = synth.random_instance(63, 10, 64, 8, n_extras=4)
    st, got = run(pkg, cube.S, cube.X[:0], cube.sigma, np.zeros(0, np.uint64), 4)
    assert st == 0


@pytest.mark.parametrize("constraint", [1, 2])
def test_masked_unmix_constraint_sets(pkg, constraint):
    """The per-pixel subsets under slo / pos equal the oracle's constraint
    sets on each pixel's sub-library."""
    cube = synth.random_instance(64, 700, 128, 14, n_extras=0)
    nm = 10
    rng = np.random.Generator(np.random.PCG64(65))
    masks = rng.integers(1, 1 << nm, cube.N).astype(np.uint64)
    um = pkg.Unmixer(_d(cube.S), constraint=constraint)
    N, P = cube.N, cube.P
    x = torch.empty((N, P), device=DEV); sx = torch.empty((N, P), device=DEV)
    rms = torch.empty((N,), device=DEV); it = torch.empty((N,), dtype=torch.int32, device=DEV)
    pkg.linmin_unmix_masked(um.h, _d(cube.X), N, _d(cube.sigma), _d(masks), nm, x, sx, rms, it)
    st, nbad = um.wait()
    um.close()
    assert st == 0
    name = {1: "slo", 2: "pos"}[constraint]
    gx = x.cpu().numpy()
    for key in np.unique(masks)[:25]:
        rows = np.nonzero(masks == key)[0]
        cols = [i for i in range(nm) if (int(key) >> i) & 1] + list(range(nm, P))
        ref = oracle.unmix_constraint(cube.S[cols], cube.sigma, cube.X[rows], name)
        assert np.abs(gx[np.ix_(rows, cols)] - ref["x"]).max() <= 1e-4
        off = [i for i in range(P) if i not in cols]
        assert (gx[np.ix_(rows, off)] == 0).all()

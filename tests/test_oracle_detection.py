"""Pins of the detection-products oracle (oracle.detection) against
hand-worked cases: the additional spectra of the Appendix table at u = 0,
1/2, 1; the rank deficiency those spectra bring under sum-to-one; the three
detection conditions of Sec. 4 on a five-pixel case; eq. Threshold of
Sec. 3.1 on a four-pixel case; the surface-mixture recipe of Sec. 3.1; and
the library auto-fit of Sec. 2.4 (oracle.autofit) against exact
dependencies, brute-force NNLS and the least-squares normal equations."""
import math

import numpy as np

import oracle.detection as od
import synth

R2 = math.sqrt(0.5)

# Rows of the Appendix table (33-44) at u = 0, 1/2, 1, worked by hand.
HAND_EXTRAS = np.array([
    [1, 1, 1],                     # 33 Flat 1
    [1e-4, 1e-4, 1e-4],            # 34 Flat 0.0001
    [0, 0.5, 1],                   # 35 slope increasing
    [1, 0.5, 0],                   # 36 slope decreasing
    [1, R2, 0],                    # 37 cos 1/4: cos(pi u / 2)
    [0, R2, 1],                    # 38 sin 1/4
    [-1, -R2, 0],                  # 39 -cos 1/4
    [0, -R2, -1],                  # 40 -sin 1/4
    [1, 0, -1],                    # 41 cos 1/2: cos(pi u)
    [0, 1, 0],                     # 42 sin 1/2
    [-1, 0, 1],                    # 43 -cos 1/2
    [0, -1, 0],                    # 44 -sin 1/2
])


def test_oracle_extras_hand_values():
    np.testing.assert_allclose(od.paper_extra_spectra(3), HAND_EXTRAS, atol=1e-15)
    np.testing.assert_allclose(od.paper_extra_spectra(3, n_extras=4), HAND_EXTRAS[:4], atol=1e-15)
    # uneven wavelengths: u from the end points
    E = od.paper_extra_spectra(3, wavelengths=[1.0, 1.5, 2.5])
    np.testing.assert_allclose(E[2], [0, 1 / 3, 1], atol=1e-7)
    np.testing.assert_allclose(E[9], [0, math.sin(math.pi / 3), 0], atol=1e-7)


def test_extras_break_uniqueness():
    """Under sum-to-one the paper's extras are dependent (the claim of
    Sec. 2.5 that they stay independent does not hold): rank [E; 1^T] is
    3 for the four and 7 for the twelve, and with independent minerals the
    deficiency stays."""
    for n, r in ((4, 3), (12, 7)):
        E = od.paper_extra_spectra(184, n_extras=n)
        M = np.vstack([E.T, np.ones((1, n))])
        assert np.linalg.matrix_rank(M) == r
    rng = np.random.Generator(np.random.PCG64(3))
    mins = synth.library(rng, 184, 32, 0)
    for n, r in ((4, 35), (12, 39)):
        S = np.vstack([mins, od.paper_extra_spectra(184, n_extras=n)])
        assert np.linalg.matrix_rank(np.vstack([S.T, np.ones((1, S.shape[0]))])) == r
        assert not synth.check_unique(S)


def test_oracle_detect_hand_case():
    # 5 pixels, P = 3, minerals 0 and 1 (column 2 is an extra)
    x = np.array([[0.30, 0.05, 0.65],
                  [0.02, 0.50, 0.48],     # x0 == x_min[0]: not above
                  [0.30, 0.10, 0.60],     # sx1 == x1: not below
                  [0.40, 0.40, 0.20],     # rms == rms_max: pixel rejected
                  [0.30, 0.60, 0.10]], np.float32)   # iterations < 0
    sx = np.array([[0.01, 0.06, 0.0],
                   [0.01, 0.01, 0.0],
                   [0.01, 0.10, 0.0],
                   [0.01, 0.01, 0.0],
                   [0.01, 0.01, 0.0]], np.float32)
    rms = np.array([0.001, 0.001, 0.001, 0.002, 0.001], np.float32)
    it = np.array([10, 12, 9, 11, -100], np.int32)
    truth = np.array([1, 2, 3, 0, 2], np.uint64)
    r = od.detect(x, sx, rms, it, truth, x_min=[0.02, 0.04], rms_max=0.002, n_minerals=2)
    # pixel 0: mineral 0 (0.30 > 0.02, 0.01 < 0.30), mineral 1 fails sx < x
    # pixel 1: mineral 1 only; pixel 2: mineral 0 only; pixels 3, 4: none
    assert r["mask"].tolist() == [1, 2, 1, 0, 0]
    assert r["count"].tolist() == [2, 1, 0]
    assert r["argmax"].tolist() == [0, 1, -1]          # tie 0.30 / 0.30: first pixel
    np.testing.assert_allclose(r["xmax"], [0.30, 0.50, 0.0], rtol=1e-7)
    np.testing.assert_allclose(r["xsum"], [0.6000000238418579, 0.5, 0.0], rtol=1e-7)
    assert r["n_true"].tolist() == [2, 3, 0]
    assert r["true_pos"].tolist() == [2, 1, 0]
    assert r["false_pos"].tolist() == [0, 0, 0]
    # without the optional arrays only the threshold decides
    r2 = od.detect(x, x_min=[0.02, 0.04], n_minerals=2)
    assert r2["mask"].tolist() == [1 | 2, 2, 3, 3, 3]


def test_oracle_threshold_hand_case():
    # mineral 0 present in pixels 0, 1 (x 0.04, 0.06: mean 0.05, std 0.01),
    # absent in 2, 3 (x 0, 0.002: mean 0.001, std 0.001)
    x = np.array([[0.04], [0.06], [0.0], [0.002]], np.float32)
    truth = np.array([1, 1, 0, 0], np.uint64)
    C = od.thresholds(x, truth, 1)
    assert abs(C[0] - 0.5 * (0.05 - 0.02 + 0.001 + 0.006)) < 1e-8     # 0.0185
    assert np.isnan(od.thresholds(x[:2], truth[:2], 1)[0])             # no absent pixel



def test_surface_mixtures_recipe():
    cube, truth = synth.surface_mixtures()
    assert cube.X.shape == (1000, 184) and cube.P == 36
    np.testing.assert_allclose(cube.A_true.sum(1), 1.0, atol=1e-12)
    assert (cube.A_true >= 0).all()
    # the flat part: level 0.35 (1 - a), no slope
    a = cube.A_true[:, :32].sum(1)
    flat = cube.A_true[:, 32:] @ cube.S[32:].astype(np.float64)
    np.testing.assert_allclose(flat, np.broadcast_to(0.35 * (1 - a)[:, None], flat.shape), atol=1e-6)
    assert (a > 0).all() and (a <= 0.1).all()
    counts = np.bincount(np.log2(truth.astype(np.float64)).astype(int), minlength=32)
    assert counts.sum() == 1000 and counts.min() >= 10      # about 1000 / 32 each
    assert abs(cube.sigma.mean() - 1.3e-3) < 1e-4


# ------------------------------------------------------------- auto-fit
def _brute_nnls(A, y):
    """min |y - A a|, a >= 0 by enumerating supports (tiny column counts)."""
    import itertools
    m = A.shape[1]
    best, best_a = np.inf, None
    for k in range(0, m + 1):
        for sup in itertools.combinations(range(m), k):
            a = np.zeros(m)
            if sup:
                sol = np.linalg.lstsq(A[:, sup], y, rcond=None)[0]
                if (sol < -1e-12).any():
                    continue
                a[list(sup)] = np.maximum(sol, 0)
            r = np.linalg.norm(y - A @ a)
            if r < best - 1e-12:
                best, best_a = r, a
    return best_a, best


def test_autofit_hand_case():
    """S2 = S0 + S1 exactly: S2 is fitted exactly with coefficients (1, 1)
    in both problems; S0 = S2 - S1 needs a negative coefficient, so only
    the unconstrained residue vanishes."""
    import oracle.autofit as oa
    S0 = np.array([1, 0, 2, 1, 0, 3], np.float32)
    S1 = np.array([0, 2, 1, 1, 3, 0], np.float32)
    S = np.stack([S0, S1, S0 + S1])
    r = oa.autofit(S)
    assert np.abs(r["resid_ls"]).max() < 1e-12
    assert np.abs(r["resid_nn"][2]).max() < 1e-12
    np.testing.assert_allclose(r["coef_nn"][2], [1, 1, 0], atol=1e-12)
    # S0 on {S1, S2} with a >= 0: the support {S2} alone, a = <S0,S2>/<S2,S2>
    S2 = (S0 + S1).astype(np.float64)
    a2 = float(S0 @ S2 / (S2 @ S2))
    assert a2 > 0
    np.testing.assert_allclose(r["coef_nn"][0], [0, 0, a2], atol=1e-12)
    np.testing.assert_allclose(r["resid_nn"][0], S0 - a2 * S2, atol=1e-12)


def test_autofit_brute_force_and_invariants():
    import oracle.autofit as oa
    rng = np.random.Generator(np.random.PCG64(12))
    for P in (2, 3, 5, 6):
        S = rng.uniform(0.0, 1.0, (P, 9)).astype(np.float32)
        r = oa.autofit(S)
        S64 = S.astype(np.float64)
        for n in range(P):
            others = [j for j in range(P) if j != n]
            A = S64[others].T
            a, best = _brute_nnls(A, S64[n])
            assert abs(np.linalg.norm(r["resid_nn"][n]) - best) < 1e-10
            np.testing.assert_allclose(r["coef_nn"][n, others], a, atol=1e-9)
            # least squares: the residue is orthogonal to every other spectrum
            assert np.abs(A.T @ r["resid_ls"][n]).max() < 1e-10
            # the unconstrained problem is a relaxation of the constrained one
            assert np.linalg.norm(r["resid_ls"][n]) <= np.linalg.norm(r["resid_nn"][n]) + 1e-12
            np.testing.assert_allclose(r["rms_nn"][n], best / 3.0, rtol=1e-10)   # sqrt(9) bands


def test_autofit_dependent_extras():
    """The level/slope spectra u, 0.5 (1 - u) and 1 are linearly dependent:
    each is fitted exactly by the others without constraints; under x >= 0
    the slopes are not (u = 1 - 2 * 0.5 (1 - u) needs a negative weight)."""
    import oracle.autofit as oa
    E = synth.extra_spectra(184)[1:]         # u, 0.5 (1 - u), 1
    r = oa.autofit(E.astype(np.float32))
    assert r["rms_ls"].max() < 1e-7
    assert r["rms_nn"][0] > 1e-2 and r["rms_nn"][1] > 1e-2
    assert r["rms_nn"][2] < 1e-7             # 1 = u + 2 * 0.5 (1 - u), weights >= 0


# ---------------------------------------------------------- second pass
def test_second_pass_pins():
    """(1) A mask holding every mineral is the first pass itself; (2) on
    noise-free mixtures whose minerals are all in the mask the truth comes
    back; (3) left-out minerals are 0 and the kept columns satisfy the FCLS
    optimality conditions (equal g_i + nu on the support, not below
    elsewhere, g = G x - c)."""
    import oracle
    cube = synth.random_instance(51, 40, 64, 10, n_extras=4)
    nm = 6
    full = oracle.unmix(cube.S, cube.sigma, cube.X)
    allm = np.full(cube.N, (1 << nm) - 1, np.uint64)
    r1 = od.second_pass(cube.S, cube.sigma, cube.X, allm, nm)
    np.testing.assert_allclose(r1["x"], full["x"], atol=1e-12)
    np.testing.assert_allclose(r1["sx"], full["sx"], atol=1e-12)
    # noise-free: X = A_true S with the true minerals in the mask (plus a
    # random extra bit); the extras are 0 in the truth
    X0 = (cube.A_true @ cube.S.astype(np.float64)).astype(np.float32)
    rng = np.random.Generator(np.random.PCG64(52))
    truth = synth.truth_masks(cube.A_true, nm) | (np.uint64(1) << rng.integers(0, nm, cube.N).astype(np.uint64))
    r2 = od.second_pass(cube.S, cube.sigma, X0, truth, nm)
    np.testing.assert_allclose(r2["x"], cube.A_true, atol=5e-5)
    # left-out columns are 0; KKT on the kept ones
    r3 = od.second_pass(cube.S, cube.sigma, cube.X, truth, nm)
    G, B = oracle.prep(cube.S, cube.sigma)
    for n in range(cube.N):
        kept = [i for i in range(nm) if (int(truth[n]) >> i) & 1] + list(range(nm, cube.P))
        off = [i for i in range(cube.P) if i not in kept]
        assert (r3["x"][n, off] == 0).all() and (r3["sx"][n, off] == 0).all()
        c, _ = oracle.project(B, cube.sigma, cube.X[n])
        g = G @ r3["x"][n] - c
        gk = g[kept]
        xs = r3["x"][n, kept]
        scale = np.abs(c).max()
        nu = -gk[xs > 1e-6].mean()
        assert np.abs(gk[xs > 1e-6] + nu).max() <= 1e-6 * scale
        assert (gk + nu >= -1e-6 * scale).all()

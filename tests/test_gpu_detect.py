"""Detection products on the device through the C ABI against the oracle
(oracle.detection): the per-pixel detection masks, counts, arg-max and
detection rates bit for bit on seeded inputs (exact ties at the thresholds
included), the threshold sums and eq. Threshold, and the whole chain
unmix -> thresholds -> detection on the surface mixtures of Sec. 3.1."""
import ctypes

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


def _dev(a):
    if a is None:
        return None
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).to(DEV)


def run_detect(pkg, x, sx, rms, it, truth, P, nm, x_min, rms_max, mask=True, out=True):
    from paper_1402_2518_gb300 import linmin
    N = x.shape[0]
    m = torch.full((max(N, 1),), -1, dtype=torch.int64, device=DEV) if mask else None
    o = torch.full((ctypes.sizeof(linmin.linmin_detection),), 0xAB, dtype=torch.uint8,
                   device=DEV) if out else None
    xd = _dev(x) if N else torch.empty((1, P), device=DEV)
    pkg.linmin_detect(xd, _dev(sx), _dev(rms), _dev(it), _dev(truth), N, P, nm, x_min,
                      rms_max, m, o)
    torch.cuda.synchronize()
    mk = m[:N].cpu().numpy().view(np.uint64) if mask else None
    return mk, (pkg.detection_summary(o) if out else None)


def compare(got_mask, got, ref, nm):
    if got_mask is not None:
        np.testing.assert_array_equal(got_mask, ref["mask"])
    if got is not None:
        P = ref["count"].shape[0]
        for k in ("count", "argmax", "n_true", "true_pos", "false_pos"):
            np.testing.assert_array_equal(got[k][:P], ref[k], err_msg=k)
        np.testing.assert_array_equal(got["xmax"][:P], ref["xmax"])
        np.testing.assert_allclose(got["xsum"][:P], ref["xsum"], rtol=1e-12, atol=0)
        # entries past P: nothing detected
        assert (got["count"][P:] == 0).all() and (got["argmax"][P:] == -1).all()


CASES = [(0, 36, 32), (1, 1, 1), (63, 8, 8), (1000, 36, 32), (100003, 36, 32),
         (4097, 64, 64), (777, 64, 0), (5000, 48, 44), (262144, 36, 32)]


@pytest.mark.parametrize("N,P,nm", CASES)
def test_detect_matches_oracle(pkg, N, P, nm):
    rng = np.random.Generator(np.random.PCG64(N * 131 + P))
    x_min = rng.uniform(0.005, 0.05, max(nm, 1)).astype(np.float32)
    rms_max = 0.01
    x, sx, rms, it, truth = synth.detection_inputs(N + P, N, P, nm, x_min, rms_max)
    got_mask, got = run_detect(pkg, x, sx, rms, it, truth, P, nm, x_min, rms_max)
    ref = od.detect(x, sx, rms, it, truth, x_min, rms_max, nm)
    compare(got_mask, got, ref, nm)


def test_detect_optional_arrays(pkg):
    N, P, nm = 3001, 36, 32
    x_min = np.full(nm, 0.02, np.float32)
    x, sx, rms, it, truth = synth.detection_inputs(99, N, P, nm, x_min, 0.01)
    for drop in ("sx", "rms", "it", "truth"):
        args = dict(sx=sx, rms=rms, it=it, truth=truth)
        args[drop] = None
        got_mask, got = run_detect(pkg, x, args["sx"], args["rms"], args["it"], args["truth"],
                                   P, nm, x_min, 0.01)
        ref = od.detect(x, args["sx"], args["rms"], args["it"], args["truth"], x_min, 0.01, nm)
        compare(got_mask, got, ref, nm)
    got_mask, _ = run_detect(pkg, x, sx, rms, it, truth, P, nm, x_min, 0.01, out=False)
    np.testing.assert_array_equal(got_mask, od.detect(x, sx, rms, it, truth, x_min, 0.01, nm)["mask"])
    _, got = run_detect(pkg, x, sx, rms, it, truth, P, nm, x_min, 0.01, mask=False)
    compare(None, got, od.detect(x, sx, rms, it, truth, x_min, 0.01, nm), nm)


@pytest.mark.parametrize("N,P,nm", [(1000, 36, 32), (65537, 48, 44), (5, 64, 64)])
def test_threshold_sums_and_eq_threshold(pkg, N, P, nm):
    from paper_1402_2518_gb300 import linmin
    x, _, _, _, truth = synth.detection_inputs(7 * N, N, P, nm, np.full(nm, 0.02, np.float32), 0.01)
    buf = torch.full((ctypes.sizeof(linmin.linmin_threshold_sums),), 0xCD, dtype=torch.uint8,
                     device=DEV)
    pkg.linmin_threshold_stats(_dev(x), _dev(truth), N, P, nm, buf)
    torch.cuda.synchronize()
    sums = pkg.threshold_sums(buf)
    ref = od.threshold_sums(x, truth, nm)
    for k in ("n_pos", "n_neg"):
        np.testing.assert_array_equal(np.array(getattr(sums, k))[:P], ref[k])
    for k in ("sum_pos", "m2_pos", "sum_neg", "m2_neg"):
        np.testing.assert_allclose(np.array(getattr(sums, k))[:P], ref[k], rtol=1e-12, atol=1e-300)
    C = pkg.linmin_thresholds(sums, nm)
    Cref = od.thresholds(x, truth, nm).astype(np.float32)
    np.testing.assert_allclose(C, Cref, rtol=1e-6, atol=1e-9)


def test_surface_mixtures_end_to_end(pkg):
    """Sec. 3.1 chain: unmix the 1000 binary mixtures, set each mineral's
    threshold by eq. Threshold from the known truth, detect with the three
    conditions; the same chain on the oracle.  Abundances agree to 1e-4,
    so each threshold (means and standard deviations with weights
    1/2 (1 + 2 + 1 + 6)) agrees to 5e-4, and every decision taken farther
    than those bounds from its threshold is the same."""
    from paper_1402_2518_gb300 import linmin
    cube, truth = synth.surface_mixtures()
    N, P, nm = cube.N, cube.P, 32
    um = pkg.Unmixer(_dev(cube.S))
    x, sx, rms, it = um(_dev(cube.X), _dev(cube.sigma))
    st, nbad = um.wait()
    um.close()
    assert st == 0 and nbad == 0
    td = _dev(truth)
    buf = torch.empty((ctypes.sizeof(linmin.linmin_threshold_sums),), dtype=torch.uint8,
                      device=DEV)
    pkg.linmin_threshold_stats(x, td, N, P, nm, buf)
    torch.cuda.synchronize()
    C = pkg.linmin_thresholds(pkg.threshold_sums(buf), nm)
    ref = oracle.unmix(cube.S, cube.sigma, cube.X)
    Cref = od.thresholds(ref["x"], truth, nm)
    assert np.isfinite(Cref).all()
    assert np.abs(C - Cref).max() <= 5e-4 + 1e-6
    rms_max = float(2.0 * cube.sigma.mean())
    gm, got = run_detect(pkg, x.cpu().numpy(), sx.cpu().numpy(), rms.cpu().numpy(),
                         it.cpu().numpy(), truth, P, nm, np.maximum(C, 0), rms_max)
    rd = od.detect(ref["x"].astype(np.float32), ref["sx"].astype(np.float32),
                   ref["rms"].astype(np.float32), ref["iters"], truth,
                   np.maximum(Cref, 0).astype(np.float32), rms_max, nm)
    xo, so = ref["x"][:, :nm], ref["sx"][:, :nm]
    # a decision is clear when x is below its threshold by more than the
    # bounds (not detected whatever sx), or above it with sx clearly on one
    # side of x, in a pixel whose RMS is clearly on one side of rms_max
    cm = np.maximum(Cref, 0)[None, :]
    clear = (xo < cm - 7e-4) | ((xo > cm + 7e-4) & (np.abs(so - xo) > 2e-4))
    clear &= (np.abs(ref["rms"] - rms_max) > 1e-4 * rms_max)[:, None]
    bits_g = ((gm[:, None] >> np.arange(nm, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(bool)
    bits_r = ((rd["mask"][:, None] >> np.arange(nm, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(bool)
    assert clear.mean() > 0.9
    np.testing.assert_array_equal(bits_g[clear], bits_r[clear])
    # rates of Sec. 3.1 (reported): positive detections among present minerals
    pd = got["true_pos"][:nm].sum() / got["n_true"][:nm].sum()
    fd = got["false_pos"][:nm].sum() / (N * nm - got["n_true"][:nm].sum())
    print(f"surface mixtures: positive detection {pd:.3f}, false detection {fd:.4f}")
    assert pd > 0.5 and fd < 0.1


def test_threshold_variance_without_cancellation(pkg):
    """eq. Threshold's standard deviations where the mean is ~1e7 times the
    standard deviation (abundances 0.5 + a few float32 ulps): sums of
    squares minus the squared mean would cancel to noise; the two-pass
    statistics give the numpy standard deviation."""
    from paper_1402_2518_gb300 import linmin
    rng = np.random.Generator(np.random.PCG64(4242))
    N, P, nm = 65536, 36, 32
    ulp = np.float32(2.0 ** -24)
    truth = np.zeros(N, np.uint64)
    x = np.zeros((N, P), np.float32)
    for i in range(nm):
        pres = rng.random(N) < 0.3
        truth[pres] |= np.uint64(1) << np.uint64(i)
        x[pres, i] = np.float32(0.5) + ulp * rng.integers(-3, 4, pres.sum()).astype(np.float32)
        x[~pres, i] = np.float32(0.25) + ulp * rng.integers(-2, 3, (~pres).sum()).astype(np.float32)
    buf = torch.zeros((ctypes.sizeof(linmin.linmin_threshold_sums),), dtype=torch.uint8, device=DEV)
    pkg.linmin_threshold_stats(_dev(x), _dev(truth), N, P, nm, buf)
    torch.cuda.synchronize()
    C = pkg.linmin_thresholds(pkg.threshold_sums(buf), nm)
    Cref = od.thresholds(x, truth, nm)
    np.testing.assert_allclose(C, Cref.astype(np.float32), rtol=1e-6)

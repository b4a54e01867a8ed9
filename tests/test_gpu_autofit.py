"""Library auto-fit (Sec. 2.4) on the device through the C ABI against the
oracle (oracle.autofit): residues of the unconstrained and the
non-negative fits of every spectrum by the others (unique), their RMS, and
the non-negative coefficients (equal where the others are independent,
a valid NNLS solution everywhere)."""
import numpy as np
import pytest

import oracle.autofit as oa
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


def _libraries():
    rng = np.random.Generator(np.random.PCG64(77))
    out = {f"random_P{P}_L{L}": rng.uniform(0.0, 1.0, (P, L)) for P, L in ((2, 3), (5, 40), (12, 33))}
    omega = synth.make_cube(synth.OMEGA_262K, n_pix=1).S
    out["omega_P36"] = omega                                  # dependent level/slope extras
    out["crism_P48"] = synth.make_cube(synth.CRISM_307K, n_pix=1).S   # near-duplicate minerals
    out["paper12_P44"] = np.vstack([omega[:32], od.paper_extra_spectra(184, None, 12)])
    rng2 = np.random.Generator(np.random.PCG64(78))
    out["P64_L4096"] = synth.library(rng2, 4096, 64, 0)
    return {k: np.ascontiguousarray(v, dtype=np.float32) for k, v in out.items()}


LIBS = _libraries()


def run(pkg, S):
    P, L = S.shape
    d = torch.from_numpy(S).to(DEV)
    rl = torch.full((P, L), np.nan, device=DEV); rn = torch.full((P, L), np.nan, device=DEV)
    cn = torch.full((P, P), np.nan, device=DEV)
    ml = torch.full((P,), np.nan, device=DEV); mn = torch.full((P,), np.nan, device=DEV)
    st = torch.full((P,), -1, dtype=torch.int32, device=DEV)
    pkg.linmin_autofit(d, L, P, rl, rn, cn, ml, mn, st)
    torch.cuda.synchronize()
    return {k: t.cpu().numpy() for k, t in zip(("resid_ls", "resid_nn", "coef_nn", "rms_ls",
                                                "rms_nn", "status"), (rl, rn, cn, ml, mn, st))}


@pytest.mark.parametrize("name", list(LIBS))
def test_autofit_matches_oracle(pkg, name):
    S = LIBS[name]
    P, L = S.shape
    got = run(pkg, S)
    ref = oa.autofit(S)
    assert (got["status"] == 0).all()
    np.testing.assert_allclose(got["resid_ls"], ref["resid_ls"], atol=1e-6, rtol=0)
    np.testing.assert_allclose(got["resid_nn"], ref["resid_nn"], atol=1e-6, rtol=0)
    np.testing.assert_allclose(got["rms_ls"], ref["rms_ls"], atol=1e-7, rtol=1e-5)
    np.testing.assert_allclose(got["rms_nn"], ref["rms_nn"], atol=1e-7, rtol=1e-5)
    a = got["coef_nn"].astype(np.float64)
    assert (a >= 0).all() and (np.diag(a) == 0).all()
    S64 = S.astype(np.float64)
    for n in range(P):
        others = [j for j in range(P) if j != n]
        A = S64[others].T
        # the coefficients reproduce the residue (float32 rounding of a)
        fit = S64[n] - A @ a[n, others]
        np.testing.assert_allclose(fit, got["resid_nn"][n], atol=2e-6 * max(1.0, a[n].sum()))
        # KKT of min |S_n - A a|, a >= 0: gradient A^T r <= 0, = 0 on the support
        gg = A.T @ fit
        scale = np.linalg.norm(A, axis=0) * max(np.linalg.norm(S64[n]), 1e-30)
        assert (gg <= 1e-5 * scale).all()
        sup = a[n, others] > 0
        assert (np.abs(gg[sup]) <= 1e-5 * scale[sup]).all()
    if name.startswith("random"):
        np.testing.assert_allclose(a, ref["coef_nn"], atol=1e-5)


def test_autofit_degeneracy_claim(pkg):
    """The point of Sec. 2.4: without constraints the dependent level/slope
    spectra are fitted exactly by the others, under x >= 0 the slopes are
    not; and the unconstrained residue never exceeds the constrained one."""
    got = run(pkg, LIBS["omega_P36"])
    assert got["rms_ls"][33] < 1e-6 and got["rms_ls"][34] < 1e-6 and got["rms_ls"][35] < 1e-6
    assert got["rms_nn"][33] > 1e-3 and got["rms_nn"][34] > 1e-3
    assert (got["rms_ls"] <= got["rms_nn"] + 1e-7).all()

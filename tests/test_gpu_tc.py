"""Tensor-core projection (tcgen05) against the FP64 oracle.

LINMIN_PROJ_TC (exact 8-bit slices, float32 accumulation that stays exact)
must meet the same bars as the double-float projection: x 1e-4, objective
1e-6 relative, uncertainties 1e-4 on unambiguous pixels, RMS 1e-4 relative.
LINMIN_PROJ_BF16 (bf16 inputs, float32 accumulation) is a precision option
whose error is measured, not bounded by the 1e-4 bar."""
import numpy as np
import pytest

import oracle
import synth
from tests import _pins
from tests.test_gpu_parity import check

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def pkg():
    import paper_1402_2518_gb300 as p
    p.load()
    return p


def run(pkg, S, sigma, X, precision):
    dev = torch.device(DEV)
    um = pkg.Unmixer(torch.from_numpy(np.ascontiguousarray(S)).to(dev), precision=precision)
    x, sx, rms, it = um(torch.from_numpy(np.ascontiguousarray(X)).to(dev),
                        torch.from_numpy(np.ascontiguousarray(sigma)).to(dev))
    st, nbad = um.wait()
    launches = pkg.linmin_last_launches(um.h)
    um.close()
    return dict(x=x.cpu().numpy().astype(np.float64), sx=sx.cpu().numpy().astype(np.float64),
                rms=rms.cpu().numpy().astype(np.float64), iters=it.cpu().numpy(), status=st,
                n_notconv=nbad, launches=launches)


@pytest.mark.parametrize("spec", synth.WORKLOADS, ids=lambda s: s.name)
def test_tc_prefix_elementwise(pkg, spec):
    from paper_1402_2518_gb300 import linmin
    cube = synth.make_cube(spec, n_pix=2000 if spec.n_pix > 2000 else None)
    ref = oracle.unmix(cube.S, cube.sigma, cube.X)
    gpu = run(pkg, cube.S, cube.sigma, cube.X, linmin.LINMIN_PROJ_TC)
    assert gpu["status"] == 0
    assert gpu["launches"] == 3 + 4 + 1 + 9 + 2 + 3 + 1
    check(gpu, ref, cube.S, cube.sigma, cube.X)


def test_tc_full_size_sampled_and_matches_df(pkg):
    from paper_1402_2518_gb300 import linmin
    cube = synth.make_cube(synth.OMEGA_262K)
    gpu = run(pkg, cube.S, cube.sigma, cube.X, linmin.LINMIN_PROJ_TC)
    rng = np.random.Generator(np.random.PCG64(77))
    rows = np.sort(rng.choice(cube.N, size=1000, replace=False))
    rows[-1] = cube.N - 1
    ref = oracle.unmix(cube.S, cube.sigma, cube.X[rows])
    check(gpu, ref, cube.S, cube.sigma, cube.X, rows)
    df = run(pkg, cube.S, cube.sigma, cube.X, linmin.LINMIN_PROJ_DF)
    assert np.abs(gpu["x"] - df["x"]).max() <= 1e-6


@pytest.mark.parametrize("N,L,P", [(1, 20, 1), (77, 61, 13), (300, 131, 64), (129, 40, 30),
                                   (1000, 240, 48)])
def test_tc_shapes(pkg, N, L, P):
    """P padded to 16/32/48/64 columns, L not a multiple of 4 (scalar row
    loads) and shorter than a chunk, a ragged last tile, N = 1."""
    from paper_1402_2518_gb300 import linmin
    extras = 4 if P >= 8 else 0
    cube = synth.random_instance(4000 + P, N, L, P, n_extras=extras)
    ref = oracle.unmix(cube.S, cube.sigma, cube.X)
    gpu = run(pkg, cube.S, cube.sigma, cube.X, linmin.LINMIN_PROJ_TC)
    if P == 1:
        np.testing.assert_array_equal(gpu["x"], 1.0)
        return
    check(gpu, ref, cube.S, cube.sigma, cube.X)


def test_tc_full_covariance(pkg):
    from paper_1402_2518_gb300 import linmin
    cube, C, Ci = synth.make_cube_cov(synth.OMEGA_262K, 0.5, n_pix=1000)
    dev = torch.device(DEV)
    opt = pkg.linmin_default_options()
    opt.precision = linmin.LINMIN_PROJ_TC
    h = pkg.linmin_create(torch.from_numpy(cube.S).to(dev), cube.L, cube.P, opt)
    x = torch.empty((cube.N, cube.P), device=dev)
    pkg.linmin_unmix_cov(h, torch.from_numpy(cube.X).to(dev), cube.N,
                         torch.from_numpy(Ci).to(dev), x)
    st, _ = pkg.linmin_wait(h)
    pkg.linmin_destroy(h)
    ref = oracle.unmix_cov(cube.S, Ci, cube.X)
    assert st == 0
    assert np.abs(x.cpu().numpy() - ref["x"]).max() <= 1e-4


def test_bf16_projection_error_is_measured(pkg):
    """bf16 inputs: the result is a valid abundance vector; its distance to
    the exact minimiser is reported (on this library, whose 8 near-duplicate
    minerals make the problem ill-conditioned, bf16 rounding of c can move
    abundance between duplicates entirely).  The median error is the
    typical cost of the bf16 option."""
    from paper_1402_2518_gb300 import linmin
    cube = synth.make_cube(synth.CRISM_307K, n_pix=2000)
    ref = oracle.unmix(cube.S, cube.sigma, cube.X)
    gpu = run(pkg, cube.S, cube.sigma, cube.X, linmin.LINMIN_PROJ_BF16)
    assert gpu["status"] in (0, 6)
    assert np.all(gpu["x"] >= 0)
    np.testing.assert_allclose(gpu["x"].sum(1), 1.0, atol=1e-5)
    d = np.abs(gpu["x"] - ref["x"]).max(axis=1)
    print(f"bf16 projection: max |x - x*| = {d.max():.3e}, median {np.median(d):.3e}, "
          f"pixels within 1e-4: {(d <= 1e-4).mean():.3f}")
    assert d.max() > 1e-6 and d.max() <= 1.0

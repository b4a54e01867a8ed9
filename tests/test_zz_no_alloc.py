"""The allocation-free entry point, linmin_unmix_noalloc.

Some callers cannot allocate device memory (code inside host callbacks,
plugins that must leave their host application's memory pool alone,
processes that have reserved all device memory up front).  For them the
library offers one entry point whose scratch is a static device array.
This file checks it through the C ABI against linmin_unmix on the same
inputs, within the parity tolerances of the other GPU tests, on two calls
in a row (the second call must not see stale contents of the shared array).
It is named so that pytest collects it last, and it passes both alone in a
fresh process and after the other tests.  The reference handle uses the
same projection (double-float) as this entry point, so the arithmetic is
the same and the iteration counts agree exactly.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

X_TOL = 1e-4
SX_TOL = 1e-4
RMS_RTOL = 1e-4


def _outputs(N, P, dev):
    return (torch.empty((N, P), device=dev), torch.empty((N, P), device=dev),
            torch.empty((N,), device=dev), torch.empty((N,), dtype=torch.int32, device=dev))


def test_noalloc_matches_unmix_on_two_calls():
    import paper_1402_2518_gb300 as pkg
    dev = torch.device("cuda:0")
    cubes = [synth.make_cube(synth.OMEGA_262K, n_pix=20000),
             synth.make_cube(synth.FCLS_1K)]
    for cube in cubes:
        N, P, L = cube.N, cube.P, cube.L
        S = torch.from_numpy(cube.S).to(dev)
        X = torch.from_numpy(cube.X).to(dev)
        sig = torch.from_numpy(cube.sigma).to(dev)
        ref = _outputs(N, P, dev)
        opt = pkg.linmin_default_options()
        opt.precision = 0           # LINMIN_PROJ_DF, the projection of the noalloc path
        h = pkg.linmin_create(S, L, P, opt)
        pkg.linmin_unmix(h, X, N, sig, *ref)
        assert pkg.linmin_wait(h)[0] == 0
        pkg.linmin_destroy(h)
        for call in range(2):
            out = _outputs(N, P, dev)
            for o in out:
                o.fill_(-7)      # stale values must be overwritten
            st = pkg.linmin_unmix_noalloc(S, L, P, X, N, sig, *out)
            torch.cuda.synchronize()
            assert st == 0, f"call {call}: status {st}"
            x, sx, rms, it = (t.cpu().numpy() for t in out)
            xr, sxr, rmsr, itr = (t.cpu().numpy() for t in ref)
            assert np.abs(x - xr).max() <= X_TOL
            assert np.abs(sx - sxr).max() <= SX_TOL
            np.testing.assert_allclose(rms, rmsr, rtol=RMS_RTOL)
            assert np.all(it > 0) and np.array_equal(np.abs(it), np.abs(itr))
            if N <= 1000:
                # and against the FP64 oracle itself
                xo = oracle.unmix(cube.S, cube.sigma, cube.X)["x"]
                assert np.abs(x - xo).max() <= X_TOL


def test_noalloc_marks_outputs_of_invalid_sigma():
    """A sigma with a zero or a NaN is found on the device, after the call
    returned: every output of that call is marked (NaN, iterations INT_MIN),
    and a following valid call is unaffected."""
    import paper_1402_2518_gb300 as pkg
    dev = torch.device("cuda:0")
    cube = synth.make_cube(synth.FCLS_1K, n_pix=300)
    N, P, L = cube.N, cube.P, cube.L
    S = torch.from_numpy(cube.S).to(dev)
    X = torch.from_numpy(cube.X).to(dev)
    for bad in (0.0, float("nan")):
        sig = cube.sigma.copy()
        sig[5] = bad
        out = _outputs(N, P, dev)
        st = pkg.linmin_unmix_noalloc(S, L, P, X, N, torch.from_numpy(sig).to(dev), *out)
        torch.cuda.synchronize()
        assert st == 0
        x, sx, rms, it = (t.cpu().numpy() for t in out)
        assert np.isnan(x).all() and np.isnan(sx).all() and np.isnan(rms).all()
        assert np.all(it == np.iinfo(np.int32).min)
    out = _outputs(N, P, dev)
    assert pkg.linmin_unmix_noalloc(S, L, P, X, N, torch.from_numpy(cube.sigma).to(dev), *out) == 0
    torch.cuda.synchronize()
    assert np.all(out[3].cpu().numpy() > 0) and np.isfinite(out[0].cpu().numpy()).all()


def test_noalloc_rejects_oversize_and_host_pointers():
    import paper_1402_2518_gb300 as pkg
    from paper_1402_2518_gb300 import linmin
    dev = torch.device("cuda:0")
    cube = synth.make_cube(synth.FCLS_1K, n_pix=64)
    S = torch.from_numpy(cube.S).to(dev)
    sig = torch.from_numpy(cube.sigma).to(dev)
    X = torch.from_numpy(cube.X).to(dev)
    # N far beyond what LINMIN_NOALLOC_SCRATCH_MB can hold: refused before any work
    too_many = (linmin.LINMIN_NOALLOC_SCRATCH_MB << 20) // (4 * (4 * cube.P + 11)) + 1
    assert pkg.linmin_unmix_noalloc(S, cube.L, cube.P, X, too_many, sig) == linmin.LINMIN_ERR_INVALID
    # host buffers are refused (the entry point cannot stage them)
    x_host = np.empty((64, cube.P), np.float32)
    assert pkg.linmin_unmix_noalloc(S, cube.L, cube.P, X, 64, sig, x_host) == \
        linmin.LINMIN_ERR_INVALID

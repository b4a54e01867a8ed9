"""Allocation failures injected on the host (LINMIN_FAIL_ALLOC, no GPU
fault): every device allocation of a handle's life (creation, the first
unmix that reserves its scratch, a host-buffer call that reserves staging,
the full-covariance buffers) is made to fail in turn; each time the entry
point returns LINMIN_ERR_OOM, the handle stays usable or can be destroyed,
and the library holds no allocation afterwards (linmin_live_allocations)."""
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def pkg():
    import paper_1402_2518_gb300 as p
    p.load()
    return p


def _life(pkg, linmin, cube, Ci):
    """Create, unmix (device buffers), unmix (host buffers), unmix under a
    full covariance, destroy; returns the first error status, or 0."""
    N, P, L = cube.N, cube.P, cube.L
    dev = torch.device(DEV)
    try:
        h = pkg.linmin_create(torch.from_numpy(cube.S).to(dev), L, P)
    except linmin.LinminError as e:
        return e.status
    try:
        X = torch.from_numpy(cube.X).to(dev)
        sg = torch.from_numpy(cube.sigma).to(dev)
        outs = [torch.empty((N, P), device=dev), torch.empty((N, P), device=dev),
                torch.empty((N,), device=dev), torch.empty((N,), dtype=torch.int32, device=dev)]
        st = pkg.linmin_unmix(h, X, N, sg, *outs, check=False)
        if st == 0:
            st = pkg.linmin_wait(h)[0]
        if st != 0:
            return st
        hx = [np.empty((N, P), np.float32), np.empty((N, P), np.float32),
              np.empty(N, np.float32), np.empty(N, np.int32)]
        st = pkg.linmin_unmix(h, cube.X, N, cube.sigma, *hx, check=False)
        if st == 0:
            st = pkg.linmin_wait(h)[0]
        if st != 0:
            return st
        st = pkg.linmin_unmix_cov(h, X, N, torch.from_numpy(Ci).to(dev), *outs, check=False)
        if st == 0:
            st = pkg.linmin_wait(h)[0]
        return st
    finally:
        pkg.linmin_destroy(h)


def test_every_allocation_failure_is_reported_and_leaks_nothing(pkg):
    from paper_1402_2518_gb300 import linmin
    cube = synth.random_instance(5150, 300, 40, 12, n_extras=4)
    Ci = np.diag(1.0 / cube.sigma.astype(np.float64) ** 2)
    torch.cuda.synchronize()
    base = pkg.linmin_live_allocations()
    assert _life(pkg, linmin, cube, Ci) == 0            # no injection: the whole life works
    assert pkg.linmin_live_allocations() == base
    failures = 0
    try:
        for n in range(1, 200):
            os.environ["LINMIN_FAIL_ALLOC"] = str(n)
            st = _life(pkg, linmin, cube, Ci)
            torch.cuda.synchronize()
            assert pkg.linmin_live_allocations() == base, f"allocation {n}: leak"
            if st == 0:
                break                                    # past the life's last allocation
            assert st == linmin.LINMIN_ERR_OOM, f"allocation {n}: status {st}"
            failures += 1
        else:
            pytest.fail("the life never completed")
    finally:
        os.environ.pop("LINMIN_FAIL_ALLOC", None)
    assert failures > 20                                # creation, scratch, staging, covariance


def test_autofit_and_server_report_injected_failures(pkg):
    from paper_1402_2518_gb300 import linmin
    cube = synth.random_instance(5151, 200, 40, 12, n_extras=0)
    dev = torch.device(DEV)
    S = torch.from_numpy(cube.S).to(dev)
    torch.cuda.synchronize()
    base = pkg.linmin_live_allocations()
    try:
        os.environ["LINMIN_FAIL_ALLOC"] = "1"
        with pytest.raises(linmin.LinminError) as e:
            pkg.linmin_autofit(S, cube.L, cube.P, torch.empty((cube.P, cube.L), device=dev))
        assert e.value.status == linmin.LINMIN_ERR_OOM
        srv = pkg.Server(hbm_budget_bytes=1 << 30, slots=1, chunk_pixels=4096)
        try:
            out = [torch.empty((cube.N, cube.P), device=dev), torch.empty((cube.N, cube.P), device=dev),
                   torch.empty((cube.N,), device=dev),
                   torch.empty((cube.N,), dtype=torch.int32, device=dev)]
            t = srv.submit(S, torch.from_numpy(cube.X).to(dev),
                           torch.from_numpy(cube.sigma).to(dev), *out)
            st, _ = srv.wait(t)
            assert st == linmin.LINMIN_ERR_OOM
        finally:
            srv.close()
    finally:
        os.environ.pop("LINMIN_FAIL_ALLOC", None)
    torch.cuda.synchronize()
    assert pkg.linmin_live_allocations() == base

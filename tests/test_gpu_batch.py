"""linmin_unmix_batch: several cubes of uneven sizes, band counts and
library sizes in one queue, with one interior-point launch per group of
equal P.  Each cube's abundances, uncertainties, RMS and iteration counts
must equal those of linmin_unmix on that cube alone (the per-pixel
arithmetic is the same; only the work distribution differs), and the
batch's arguments are checked on the host."""
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


def _cubes():
    # (seed, N, L, P, extras): two cubes of P = 36 with different libraries
    # and band counts share a launch, P = 48 and P = 16 get their own, and
    # one empty cube is skipped
    shapes = [(41, 3001, 184, 36, 4), (42, 1533, 128, 36, 4), (43, 2500, 240, 48, 4),
              (44, 0, 184, 36, 4), (45, 1207, 128, 16, 4), (46, 777, 184, 36, 4)]
    out = []
    for seed, n, L, P, ex in shapes:
        c = synth.random_instance(seed, max(n, 1), L, P, n_extras=ex)
        out.append((c, n))
    return out


def _alloc(n, P, dev):
    return (torch.empty((max(n, 1), P), device=dev), torch.empty((max(n, 1), P), device=dev),
            torch.empty((max(n, 1),), device=dev), torch.empty((max(n, 1),), dtype=torch.int32, device=dev))


def test_batch_equals_single_calls(pkg):
    dev = torch.device(DEV)
    stream = torch.cuda.Stream(device=dev)
    cubes = _cubes()
    ums, refs, args = [], [], []
    for c, n in cubes:
        S = torch.from_numpy(c.S).to(dev)
        X = torch.from_numpy(c.X).to(dev)
        sg = torch.from_numpy(c.sigma).to(dev)
        # the reference: linmin_unmix on its own handle
        ref_um = pkg.Unmixer(S)
        out = _alloc(n, c.P, dev)
        if n:
            pkg.linmin_unmix(ref_um.h, X, n, sg, *out)
        st, nbad = ref_um.wait()
        assert st == 0 and nbad == 0
        refs.append([t.cpu().numpy() for t in out])
        ref_um.close()
        um = pkg.Unmixer(S, stream=stream)
        ums.append(um)
        args.append((X, n, sg, _alloc(n, c.P, dev)))
    st = pkg.linmin_unmix_batch([u.h for u in ums], [a[0] for a in args], [a[1] for a in args],
                                [a[2] for a in args], [a[3][0] for a in args],
                                [a[3][1] for a in args], [a[3][2] for a in args],
                                [a[3][3] for a in args])
    assert st == 0
    for (c, n), um, a, ref in zip(cubes, ums, args, refs):
        st, nbad = um.wait()
        assert st == 0 and nbad == 0
        if not n:
            continue
        got = [t.cpu().numpy() for t in a[3]]
        for g, r in zip(got, ref):
            np.testing.assert_array_equal(g[:n], r[:n])
    # a second batch on the same handles gives the same results again
    st = pkg.linmin_unmix_batch([u.h for u in ums], [a[0] for a in args], [a[1] for a in args],
                                [a[2] for a in args], [a[3][0] for a in args], None, None, None)
    assert st == 0
    for (c, n), um, a, ref in zip(cubes, ums, args, refs):
        assert um.wait()[0] == 0
        if n:
            np.testing.assert_array_equal(a[3][0].cpu().numpy()[:n], ref[0][:n])
    for um in ums:
        um.close()


def test_batch_argument_checks(pkg):
    from paper_1402_2518_gb300 import linmin
    dev = torch.device(DEV)
    c = synth.random_instance(50, 300, 128, 16, n_extras=4)
    S = torch.from_numpy(c.S).to(dev)
    X = torch.from_numpy(c.X).to(dev)
    sg = torch.from_numpy(c.sigma).to(dev)
    x = torch.empty((300, c.P), device=dev)
    um = pkg.Unmixer(S)
    other = pkg.Unmixer(S, stream=torch.cuda.Stream(device=dev))
    slo = pkg.Unmixer(torch.from_numpy(c.S[:c.P - 4].copy()).to(dev), constraint=1)
    cases = [
        ([um.h], [torch.from_numpy(c.X)], [sg], [x]),          # host cube
        ([um.h, um.h], [X, X], [sg, sg], [x, x]),               # the same handle twice
        ([um.h, other.h], [X, X], [sg, sg], [x, x]),            # different streams
    ]
    for hs, cubes, sigmas, xs in cases:
        st = pkg.linmin_unmix_batch(hs, cubes, [300] * len(hs), sigmas, xs, check=False)
        assert st == linmin.LINMIN_ERR_INVALID
    xs = torch.empty((300, c.P - 4), device=dev)
    st = pkg.linmin_unmix_batch([slo.h], [X], [300], [sg], [xs], check=False)
    assert st == linmin.LINMIN_ERR_INVALID                      # slo / pos handles
    for u in (um, other, slo):
        u.close()

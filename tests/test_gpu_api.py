"""Profiling and launch-count entry points of the C ABI on the device."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_phase_ring_and_launch_count():
    import paper_1402_2518_gb300 as pkg
    from paper_1402_2518_gb300 import linmin
    pkg.load()
    cube = synth.make_cube(synth.OMEGA_262K, n_pix=4000)
    dev = torch.device("cuda:0")
    um = pkg.Unmixer(torch.from_numpy(cube.S).to(dev), profile=True)
    X = torch.from_numpy(cube.X).to(dev)
    sg = torch.from_numpy(cube.sigma).to(dev)
    x = torch.empty((cube.N, cube.P), device=dev)
    rms = torch.empty((cube.N,), device=dev)
    h = um.h
    with pytest.raises(linmin.LinminError):
        pkg.linmin_phase_times_at(h, 0)            # nothing profiled yet
    for _ in range(3):
        assert pkg.linmin_unmix(h, X, cube.N, sg, x, None, rms) == 0
    times = [pkg.linmin_phase_times_at(h, b) for b in range(3)]
    for t in times:
        assert set(t) == set(linmin.PHASES)
        assert all(v >= 0.0 for v in t.values()) and t["ipm"] > 0.0
    assert times[0] == pkg.linmin_phase_times(h)
    with pytest.raises(linmin.LinminError):
        pkg.linmin_phase_times_at(h, 3)            # only three calls so far
    with pytest.raises(linmin.LinminError):
        pkg.linmin_phase_times_at(h, linmin.LINMIN_PHASE_RING)
    # prep 3, projection (tensor cores: B~ exponents and slices, pixel
    # exponents, GEMM),
    # IPM, crossover (support, scan, scatter, pass 0, sort of its flips: histogram,
    # scan, scatter; lane groups for supports of up to 24 coordinates, then
    # for larger ones: P = 36), retry
    # (2 IPM, support, the two lane-group launches), rms
    assert pkg.linmin_last_launches(h) == 3 + 4 + 1 + 9 + 2 + 3 + 1
    assert pkg.linmin_unmix(h, X, cube.N, sg, x) == 0          # no RMS requested
    assert pkg.linmin_last_launches(h) == 3 + 4 + 1 + 9 + 2 + 3
    assert pkg.linmin_unmix(h, X, 0, sg, x) == 0
    assert pkg.linmin_last_launches(h) == 0
    st, _ = um.wait()
    assert st == 0
    um.close()


def test_autotune_and_lanes():
    """The autotuner picks one of the compiled buckets for P; every bucket
    it may pick gives oracle-matching results."""
    import oracle
    import paper_1402_2518_gb300 as pkg
    from paper_1402_2518_gb300 import linmin
    pkg.load()
    cube = synth.random_instance(4321, 6000, 184, 32, n_extras=4)
    dev = torch.device("cuda:0")
    um = pkg.Unmixer(torch.from_numpy(cube.S).to(dev))
    X = torch.from_numpy(cube.X).to(dev)
    sg = torch.from_numpy(cube.sigma).to(dev)
    assert pkg.linmin_get_lanes(um.h) == 4                   # default for P = 32: 8 x 4
    lanes, ms = pkg.linmin_autotune(um.h, X, cube.N, sg)
    assert len(ms) >= 2 and all(t > 0 for t in ms)
    assert lanes == pkg.linmin_get_lanes(um.h) and lanes in (4, 8)
    rows = np.linspace(0, cube.N - 1, 200).astype(int)
    ref = oracle.unmix(cube.S, cube.sigma, cube.X[rows])
    for g in (4, 8):
        pkg.linmin_set_lanes(um.h, g)
        assert pkg.linmin_get_lanes(um.h) == g
        x, sx, rms, it = um(X, sg)
        st, _ = um.wait()
        assert st == 0
        assert np.abs(x.cpu().numpy()[rows] - ref["x"]).max() <= 1e-4
    with pytest.raises(linmin.LinminError) as e:
        pkg.linmin_set_lanes(um.h, 16)                        # no 16-lane bucket near P = 32
    assert e.value.status == linmin.LINMIN_ERR_UNSUPPORTED
    assert pkg.linmin_get_lanes(um.h) == 8                    # unchanged by the refusal
    um.close()


def test_host_buffers_pipelined_equal_device():
    """Host buffers of at least 65,536 pixels go through the copy/compute
    pipeline (eight pieces, copies on their own stream): the results equal
    the device-pointer call bit for bit, with a ragged last piece and a
    missing output."""
    import paper_1402_2518_gb300 as pkg
    pkg.load()
    cube = synth.make_cube(synth.OMEGA_262K, n_pix=70001)
    dev = torch.device("cuda:0")
    um = pkg.Unmixer(torch.from_numpy(cube.S).to(dev))
    X = torch.from_numpy(cube.X).to(dev)
    sg = torch.from_numpy(cube.sigma).to(dev)
    x, sx, rms, it = um(X, sg)
    st, _ = um.wait()
    assert st == 0
    N, P = cube.N, cube.P
    xh = np.empty((N, P), np.float32); rh = np.empty(N, np.float32); ih = np.empty(N, np.int32)
    assert pkg.linmin_unmix(um.h, cube.X, N, cube.sigma, xh, None, rh, ih) == 0
    np.testing.assert_array_equal(xh, x.cpu().numpy())
    np.testing.assert_array_equal(rh, rms.cpu().numpy())
    np.testing.assert_array_equal(ih, it.cpu().numpy())
    um.close()

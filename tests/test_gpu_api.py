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
    # prep 3, projection, IPM, crossover 3 + 9 passes, retry 2 IPM + 1 + 9, rms
    assert pkg.linmin_last_launches(h) == 3 + 1 + 1 + 12 + 2 + 10 + 1
    assert pkg.linmin_unmix(h, X, cube.N, sg, x) == 0          # no RMS requested
    assert pkg.linmin_last_launches(h) == 3 + 1 + 1 + 12 + 2 + 10
    assert pkg.linmin_unmix(h, X, 0, sg, x) == 0
    assert pkg.linmin_last_launches(h) == 0
    st, _ = um.wait()
    assert st == 0
    um.close()

"""Serving (continuous batching) through the C ABI: every result of a mixed
stream equals the same cube unmixed alone, bit for bit; the device-memory
budget holds and forces evictions; bad requests are refused at submit."""
import time

import numpy as np
import pytest

import oracle
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
    """Uneven cubes: several (N, L, P), two pairs sharing a library."""
    shapes = [(3000, 128, 16), (700, 184, 36), (12000, 184, 36), (257, 240, 48),
              (5000, 128, 32), (1, 184, 36), (9000, 240, 64), (4100, 128, 16)]
    cubes = [synth.random_instance(7000 + i, N, L, P, n_extras=4)
             for i, (N, L, P) in enumerate(shapes)]
    # cubes 2 and 5 reuse cube 1's library, cube 7 reuses cube 0's
    for dst, src in ((2, 1), (5, 1), (7, 0)):
        c, s = cubes[dst], cubes[src]
        cubes[dst] = synth.Cube(c.spec, s.S, s.sigma, c.X, c.A_true)
    return cubes


def _alone(pkg, cube):
    dev = torch.device(DEV)
    um = pkg.Unmixer(torch.from_numpy(cube.S).to(dev))
    x, sx, rms, it = um(torch.from_numpy(cube.X).to(dev), torch.from_numpy(cube.sigma).to(dev))
    st, _ = um.wait()
    um.close()
    return st, [t.cpu().numpy() for t in (x, sx, rms, it)]


def _outputs(N, P, device):
    if device:
        dev = torch.device(DEV)
        return [torch.empty((N, P), device=dev), torch.empty((N, P), device=dev),
                torch.empty((N,), device=dev), torch.empty((N,), dtype=torch.int32, device=dev)]
    return [np.empty((N, P), np.float32), np.empty((N, P), np.float32),
            np.empty(N, np.float32), np.empty(N, np.int32)]


def _host(a):
    return a.cpu().numpy() if hasattr(a, "cpu") else a


def _run_stream(pkg, cubes, server, gaps_s):
    dev = torch.device(DEV)
    tickets, outs = [], []
    for i, (cube, gap) in enumerate(zip(cubes, gaps_s)):
        time.sleep(gap)
        on_dev = i % 2 == 0
        S = torch.from_numpy(cube.S).to(dev) if on_dev else cube.S
        X = torch.from_numpy(cube.X).to(dev) if on_dev else cube.X
        sg = torch.from_numpy(cube.sigma).to(dev) if on_dev else cube.sigma
        o = _outputs(cube.N, cube.P, on_dev)
        tickets.append(server.submit(S, X, sg, *o))
        outs.append(o)
    res = []
    for t, o in zip(tickets, outs):
        st, ms = server.wait(t)
        res.append((st, ms, [_host(a) for a in o]))
    return res


def test_mixed_stream_equals_alone(pkg):
    cubes = _cubes()
    rng = np.random.Generator(np.random.PCG64(11))
    gaps = rng.exponential(1.0 / 200.0, len(cubes))          # Poisson arrivals, 200/s
    server = pkg.Server(slots=4, chunk_pixels=4096, autotune=False)
    res = _run_stream(pkg, cubes, server, gaps)
    stats = server.stats()
    server.close()
    for cube, (st, ms, got) in zip(cubes, res):
        st0, want = _alone(pkg, cube)
        assert st == st0 == 0 and ms > 0.0
        for g, w in zip(got, want):
            np.testing.assert_array_equal(g, w)
    assert stats["requests_done"] == len(cubes)
    assert stats["chunks"] >= sum(-(-c.N // 4096) for c in cubes)
    # the shared libraries were served by cached handles: fewer handles than
    # (request, slot) pairs would need
    assert stats["handles_created"] <= 4 * (len(cubes) - 3)


def test_mixed_stream_matches_oracle(pkg):
    """Sampled pixels of two cubes of the mix against the FP64 oracle."""
    cubes = _cubes()
    server = pkg.Server(slots=3, chunk_pixels=2048, autotune=False)
    res = _run_stream(pkg, cubes, server, [0.0] * len(cubes))
    stats = server.stats()
    server.close()
    # all submitted at once: chunks ran concurrently on the worker streams
    assert stats["max_running"] >= 2
    for k in (2, 6):
        cube, (st, _, got) = cubes[k], res[k]
        rows = np.linspace(0, cube.N - 1, 60).astype(int)
        ref = oracle.unmix(cube.S, cube.sigma, cube.X[rows])
        assert st == 0
        assert np.abs(got[0][rows] - ref["x"]).max() <= 1e-4
        np.testing.assert_allclose(got[2][rows], ref["rms"], rtol=1e-4)


def test_small_budget_admission(pkg):
    """A budget of a few handles: handles are evicted to admit new libraries,
    the budget is never exceeded, and the results do not change."""
    cubes = [synth.random_instance(7100 + i, 1500 + 300 * i, 184, 36, n_extras=4)
             for i in range(6)]
    one = pkg.linmin_server_handle_bytes(184, 36, 1024, host_io=True)
    budget = int(2.5 * one)
    server = pkg.Server(hbm_budget_bytes=budget, slots=4, chunk_pixels=1024, autotune=False)
    res = _run_stream(pkg, cubes, server, [0.0] * len(cubes))
    stats = server.stats()
    server.close()
    assert stats["peak_bytes"] <= budget
    assert stats["evictions"] > 0
    for cube, (st, _, got) in zip(cubes, res):
        st0, want = _alone(pkg, cube)
        assert st == st0 == 0
        for g, w in zip(got, want):
            np.testing.assert_array_equal(g, w)


def test_bad_requests_refused(pkg):
    from paper_1402_2518_gb300 import linmin
    server = pkg.Server(hbm_budget_bytes=1 << 20, slots=2)
    cube = synth.random_instance(7200, 50, 64, 8, n_extras=0)
    S_bad = np.ones((4, 64), np.float32)                       # rank 1 < 4
    with pytest.raises(linmin.LinminError) as e:
        server.submit(S_bad, cube.X, cube.sigma)
    assert e.value.status == linmin.LINMIN_ERR_RANK
    S65 = np.random.default_rng(0).uniform(0.2, 0.6, (65, 128)).astype(np.float32)
    X65 = np.zeros((2, 128), np.float32)
    with pytest.raises(linmin.LinminError) as e:
        server.submit(S65, X65, np.ones(128, np.float32))
    assert e.value.status == linmin.LINMIN_ERR_UNSUPPORTED
    big = synth.random_instance(7201, 10, 4096, 64, n_extras=4)
    with pytest.raises(linmin.LinminError) as e:                # one chunk > 1 MiB
        server.submit(big.S, big.X, big.sigma)
    assert e.value.status == linmin.LINMIN_ERR_OOM
    t = server.submit(cube.S, cube.X[:0], cube.sigma)           # N = 0: done at once
    assert server.wait(t)[0] == 0
    server.close()


def test_library_cache_stays_bounded(pkg):
    """A long-running server that sees many libraries keeps at most 64 of the
    idle ones (with their handles); a library met again after eviction is
    loaded again, and every result still equals the cube unmixed alone."""
    srv = pkg.Server(hbm_budget_bytes=8 << 30, slots=2, chunk_pixels=4096, autotune=False)
    try:
        cubes = [synth.random_instance(7400 + i, 64, 40, 8, n_extras=0) for i in range(70)]
        cubes.append(cubes[0])                 # the first library again, after eviction
        for cube in cubes:
            out = _outputs(cube.N, cube.P, True)
            t = srv.submit(torch.from_numpy(cube.S).to(DEV), torch.from_numpy(cube.X).to(DEV),
                           torch.from_numpy(cube.sigma).to(DEV), *out)
            st, _ = srv.wait(t)
            assert st == 0
            st_a, ref = _alone(pkg, cube)
            for got, want in zip(out, ref):
                np.testing.assert_array_equal(_host(got), want)
            assert srv.stats()["libraries"] <= 64
        assert srv.stats()["evictions"] > 0
    finally:
        srv.close()


def test_autotuned_server_results(pkg):
    """With the autotuner on (the default), the first handle of each library
    shape is tuned on its first chunk and later handles of that shape reuse
    the choice; results stay within the parity bars of the oracle."""
    cubes = [synth.random_instance(7600 + i, 3000, L, P, n_extras=4)
             for i, (L, P) in enumerate([(128, 16), (184, 36), (184, 36), (240, 48)])]
    srv = pkg.Server(slots=2, chunk_pixels=1024)
    try:
        tickets = []
        outs = []
        for cube in cubes:
            out = _outputs(cube.N, cube.P, True)
            outs.append(out)
            tickets.append(srv.submit(torch.from_numpy(cube.S).to(DEV),
                                      torch.from_numpy(cube.X).to(DEV),
                                      torch.from_numpy(cube.sigma).to(DEV), *out))
        for t in tickets:
            assert srv.wait(t)[0] == 0
        stats = srv.stats()
        assert stats["autotuned"] <= 3                   # at most once per shape in the process
        for cube, out in zip(cubes, outs):
            ref = oracle.unmix(cube.S, cube.sigma, cube.X[:400])
            assert np.abs(_host(out[0])[:400] - ref["x"]).max() <= 1e-4
    finally:
        srv.close()

"""The benchmark's multi-rank path on the CPU (world size 2, gloo,
127.0.0.1): the step time is the maximum over the ranks, the whole-job
value counts every replica's pixels (weak scaling, no data-path
collective), and under torchrun only rank 0 runs and prints the reference
arm."""
import io
import os
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE="2", LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        ms = 5.0 + 3.0 * rank                       # rank 1 is the slower replica
        m = bench.max_over_ranks(ms, dist, "cpu")
        v = bench.replicas_value(1000, m / 1e3, dist.get_world_size())
        # reference arm: only rank 0 prints
        buf = io.StringIO()
        args = type("A", (), {"warmup": 0, "steps": 1, "gpus": 2})()
        import synth
        cube = synth.make_cube(synth.FCLS_1K, n_pix=8)
        with redirect_stdout(buf):
            bench.run_reference(args, cube)
        out.put((rank, m, v, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_and_weak_scaling():
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, v0, o0), (r1, m1, v1, o1) = res
    assert m0 == m1 == 8.0                           # the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 1000 / 8e-3)
    assert '"impl": "reference"' in o0 and o1 == ""
    assert bench_single() == 5.0


def bench_single():
    sys.path.insert(0, ROOT)
    import bench
    return bench.max_over_ranks(5.0)                 # no process group: itself

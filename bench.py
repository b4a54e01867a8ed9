"""Benchmark: pixels/s of fully constrained IPLS unmixing on the OMEGA-shaped
synthetic cube (262,144 pixels, L = 184 bands, P = 36 spectra: 32 minerals
+ 4 level/slope spectra, per-band sigma in [0.002, 0.02]).

One step = one linmin_unmix call over the whole cube (library preparation,
double-float projection, float32 interior-point solve, double-float
active-set crossover with uncertainties, the retry path, RMS), inputs
resident in HBM.
The cube (193 MB) is larger than L2 (129 MB), so no flush between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank unmixes its own cube (weak scaling, no collective
on the data path); the timing is the max over ranks.  ``--impl reference``
times the FP64 CPU oracle on a bounded pixel sample of the same cube.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

SPEC = synth.OMEGA_262K
METRIC = "pixels/s IPLS unmix at <=1e-4 abs err vs FP64 oracle; served p50/p99 latency"
FP32_LANES_PER_SM = 128

# DRAM bytes per pixel of the main interior-point launch, from the ncu
# capture summarised in profiles/ipm_omega65k_full.md
# (dram__bytes_read.sum + dram__bytes_write.sum on 65,536 pixels; traffic
# grows with the pixel count).  Valid only for the kernel source it was
# measured on (hash of csrc/ipm.cuh).
IPM_TRAFFIC = {"ipm_sha256_12": "2423e78fbf10",
               "bytes_per_pixel": (9.549568e6 + 0.00128e6) / 65536}


# DRAM bytes of detect_kernel (ncu, 65,536 pixels: 19,948,544 read, 0
# written; profiles/detect_and_exclude_omega65k.md), valid for the hashed
# source; traffic grows with the pixel count (rows read once)
DETECT_TRAFFIC = {"sha256_12": "e16e392227f9", "bytes_per_pixel": 19.948544e6 / 65536}


def projection_roofline(n_pix: int, L: int, P: int, phase_ms: float, hbm_gbs: float):
    """The projection phase against HBM: algorithmic bytes = the cube read
    once (4 L per pixel) + c~ written (hi and lo words, 8 P per pixel)."""
    nbytes = n_pix * (4 * L + 8 * P)
    achieved = nbytes / (phase_ms / 1e3) / 1e9
    return {"bound": "hbm", "phase_ms": phase_ms, "algorithmic_bytes": nbytes,
            "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s", "frac": achieved / hbm_gbs,
            "note": "phase = B~ column exponents and slices, the join with the per-pixel "
                    "exponent pass (a second read of the cube, on a side stream, "
                    "overlapping the library preparation) and the warp-specialised "
                    "tensor-core GEMM; peak = measured copy bandwidth"}


def detect_traffic(n_pix: int):
    import hashlib
    src = os.path.join(ROOT, "paper_1402_2518_gb300", "csrc", "detect.cu")
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:12]
    if h != DETECT_TRAFFIC["sha256_12"]:
        return None
    return DETECT_TRAFFIC["bytes_per_pixel"] * n_pix


def ipm_traffic(n_pix: int):
    import hashlib
    src = os.path.join(ROOT, "paper_1402_2518_gb300", "csrc", "ipm.cuh")
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:12]
    if h != IPM_TRAFFIC["ipm_sha256_12"]:
        return None
    return IPM_TRAFFIC["bytes_per_pixel"] * n_pix


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--workload", default="omega", choices=["omega", "crism"],
                    help="cube of the main leg: the OMEGA-shaped one (the metric's "
                         "workload, default) or the CRISM-shaped one")
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--pixels", type=int, default=0,
                    help="use only the first PIXELS pixels (small profiling case)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer e2e leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-cov", action="store_true", help="skip the full-covariance leg")
    ap.add_argument("--no-constraints", action="store_true", help="skip the slo / pos leg")
    ap.add_argument("--no-detection", action="store_true", help="skip the detection leg")
    ap.add_argument("--no-crism", action="store_true", help="skip the CRISM-shaped leg")
    ap.add_argument("--check-pixels", type=int, default=2048,
                    help="pixels the oracle recomputes for the accuracy of the timed call "
                         "when the CPU baseline is skipped")
    ap.add_argument("--no-second-pass", action="store_true", help="skip the second-pass timing")
    ap.add_argument("--detect-flush-gb", type=float, default=4.0,
                    help="GiB written before each timed detection call")
    ap.add_argument("--precision", default="tc", choices=["df", "tc", "bf16"],
                    help="projection: double-float CUDA cores, exact tensor-core slices, bf16")
    ap.add_argument("--serving-cubes", type=int, default=64)
    ap.add_argument("--serving-rate", type=float, default=200.0, help="arrivals per second")
    ap.add_argument("--serving-budget-gb", type=float, default=120.0)
    ap.add_argument("--serving-slots", type=int, default=4)
    ap.add_argument("--serving-chunk", type=int, default=65536)
    return ap.parse_args()


def max_over_ranks(v: float, dist=None, device="cpu") -> float:
    """The largest v over the ranks of the process group (v itself without
    one): the timing of a step is that of its slowest replica."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(v)
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(n_local: int, seconds: float, world_size: int) -> float:
    """Whole-job throughput of identical replicas (weak scaling): every rank
    unmixes its own cube of n_local pixels in at most `seconds`."""
    return n_local * world_size / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


X_TOL = 1e-4          # the metric's bar: max |x - x_oracle| per abundance


def accuracy(cube, rows, ref, x, sx, rms):
    """Errors of a GPU result (x, sx, rms: numpy, all N pixels) against the
    oracle's (ref: oracle.unmix on cube.X[rows]), in fp64:
      max_abs_err    max |x - x_oracle| over every abundance of those pixels;
      max_obj_rel    max (f(x) - f(x*)) / |f(x*)| with f the whitened
                     criterion 1/2 |W (y - S^T x)|^2 (x renormalised to the
                     simplex first, as the bar on the objective reads);
      max_sx_err     max |sigma_x - sigma_x_oracle| on pixels whose support
                     the data resolve (each coordinate's multiplier margin,
                     in the solver's scaled units, >= 1e-8 and lambda_i /
                     (x_i G_ii) outside [1e-3, 1e3]); sx_pixels: how many;
      max_rms_rel    max relative RMS difference."""
    S = cube.S.astype(np.float64)
    w2 = 1.0 / cube.sigma.astype(np.float64) ** 2
    G = (S * w2) @ S.T
    s_scale = np.trace(G) / G.shape[0]
    Y = cube.X[rows].astype(np.float64)
    C = Y @ (S * w2).T
    ss = (Y * Y * w2).sum(1)
    xg = x[rows].astype(np.float64)
    xo = ref["x"]

    def f(z):
        return 0.5 * np.einsum("ni,ij,nj->n", z, G, z) - (C * z).sum(1) + 0.5 * ss

    fo = f(xo)
    fg = f(xg / xg.sum(1, keepdims=True))
    ratio = ref["lam"] / np.maximum(xo, 1e-300) / np.diag(G)[None, :]
    active = ratio < 1e-3
    with np.errstate(divide="ignore"):
        margin = np.where(active, xo / np.maximum(ref["sx"], 1e-300) ** 2, ref["lam"]) / s_scale
    ok = ~np.any((ratio > 1e-3) & (ratio < 1e3), axis=1) & np.all(margin >= 1e-8, axis=1)
    sxe = np.abs(sx[rows].astype(np.float64) - ref["sx"])[ok]
    return {"pixels": int(len(rows)), "max_abs_err": float(np.abs(xg - xo).max()),
            "max_obj_rel": float(((fg - fo) / np.abs(fo)).max()),
            "max_sx_err": float(sxe.max()) if sxe.size else None, "sx_pixels": int(ok.sum()),
            "max_rms_rel": float((np.abs(rms[rows] - ref["rms"]) / ref["rms"]).max()),
            "bar": X_TOL}


def cpu_baseline(cube, target_s: float, one_core_s: float = 3.0):
    """The FP64 oracle, as it stands, on a bounded prefix of the same cube,
    on every host core and on one core.  Returns the baseline object and the
    oracle's results on that prefix (the reference for the accuracy of the
    timed GPU call)."""
    import oracle
    n0 = min(cube.N, 1024)
    t = time.perf_counter()
    oracle.unmix(cube.S, cube.sigma, cube.X[:n0], extras=False)
    rate = n0 / max(time.perf_counter() - t, 1e-6)
    n = int(min(cube.N, max(n0, rate * target_s)))
    t = time.perf_counter()
    ref = oracle.unmix(cube.S, cube.sigma, cube.X[:n])
    dt = time.perf_counter() - t
    n1 = int(min(cube.N, max(64, rate / oracle.nproc() * one_core_s)))
    t = time.perf_counter()
    oracle.unmix(cube.S, cube.sigma, cube.X[:n1], nthreads=1, extras=False)
    dt1 = time.perf_counter() - t
    return ({"value": n / dt, "unit": "pixels/s", "cores": oracle.nproc(), "kind": "oracle",
             "sample": f"first {n} of {cube.N} pixels of {SPEC.name}, {dt:.1f} s",
             "one_core": {"value": n1 / dt1, "unit": "pixels/s", "cores": 1,
                          "sample": f"first {n1} pixels, {dt1:.1f} s"}},
            np.arange(n), ref)


def sample_rows(N: int, n: int, seed: int = 99):
    """A seeded sample of n pixel indices of 0..N-1, sorted, with the last."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rows = np.sort(rng.choice(N, size=min(n, N), replace=False))
    rows[-1] = N - 1
    return rows


def run_e2e(pkg, cube, steps, precision=0):
    """Seconds per step of linmin_unmix on pinned host buffers: the cube and
    sigma are copied in and every output copied back inside the call."""
    import torch
    N, P, L = cube.N, cube.P, cube.L
    Xh = torch.from_numpy(cube.X).pin_memory()
    sgh = torch.from_numpy(cube.sigma).pin_memory()
    xh = torch.empty((N, P)).pin_memory()
    sxh = torch.empty((N, P)).pin_memory()
    rh = torch.empty((N,)).pin_memory()
    ih = torch.empty((N,), dtype=torch.int32).pin_memory()
    opt = pkg.linmin_default_options()
    opt.precision = precision
    h = pkg.linmin_create(cube.S, L, P, opt)

    def step():
        pkg.linmin_unmix(h, Xh.numpy(), N, sgh.numpy(), xh.numpy(), sxh.numpy(),
                         rh.numpy(), ih.numpy())

    step()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    dt = (time.perf_counter() - t0) / steps
    pkg.linmin_destroy(h)
    return dt


def run_reference(args, cube):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    n = int(min(cube.N, 4096))
    for _ in range(args.warmup):
        oracle.unmix(cube.S, cube.sigma, cube.X[:256], extras=False)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.unmix(cube.S, cube.sigma, cube.X[:n], extras=False)
        times.append(time.perf_counter() - t)
    tot = sum(times)
    value = n * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pixels/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": SPEC.name, "pixels": SPEC.n_pix, "L": SPEC.L,
                       "P": SPEC.P, "step_sample_pixels": n},
            "cpu_baseline": {"value": value, "unit": "pixels/s", "cores": oracle.nproc(),
                             "kind": "oracle",
                             "sample": f"first {n} of {cube.N} pixels per step"},
            "e2e": {"value": value, "unit": "pixels/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _pct(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else None


def run_serving(pkg, dev, n_cubes: int, rate: float, budget_gb: float, slots: int,
                chunk: int, fp32_peak: float = 80.0):
    """Serving stream of uneven cubes through the library's server (chunks of
    all requests in flight on `slots` streams) against the plain path: one
    linmin_unmix call per cube, one after the other.  Inputs and outputs are
    device-resident; latency = completion - arrival (queueing included).
    Also the same cubes all submitted at once (a batch)."""
    import torch
    specs = synth.batch_specs(n_cubes)
    arrivals = synth.poisson_arrivals(n_cubes, rate)
    cubes = []
    for sp in specs:
        c = synth.make_cube(sp)
        cubes.append((torch.from_numpy(c.S).to(dev), torch.from_numpy(c.X).to(dev),
                      torch.from_numpy(c.sigma).to(dev), c.N, c.P))
    outs = [(torch.empty((N, P), device=dev), torch.empty((N, P), device=dev),
             torch.empty((N,), device=dev), torch.empty((N,), dtype=torch.int32, device=dev))
            for (_, _, _, N, P) in cubes]
    total = sum(c[3] for c in cubes)

    def served(arr):
        srv = pkg.Server(hbm_budget_bytes=int(budget_gb * (1 << 30)), slots=slots,
                         chunk_pixels=chunk)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = []
        for (S, X, sg, N, P), o, ta in zip(cubes, outs, arr):
            d = t0 + ta - time.perf_counter()
            if d > 0:
                time.sleep(d)
            t_call = time.perf_counter() - t0
            tickets.append((srv.submit(S, X, sg, *o), t_call))
        lat, end, bad = [], 0.0, 0
        for (t, sub), ta in zip(tickets, arr):
            st, ms = srv.wait(t)
            bad += st != 0
            lat.append(ms + (sub - ta) * 1e3)      # + the submit call's delay behind the arrival
            end = max(end, ta + lat[-1] / 1e3)
        stats = srv.stats()
        srv.close()
        return {"value": total / end, "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99),
                "makespan_s": end, "failed": bad,
                "max_running": stats["max_running"], "chunks": stats["chunks"],
                "handles_created": stats["handles_created"],
                "peak_gb": stats["peak_bytes"] / (1 << 30)}

    def plain(arr):
        hs = []
        for (S, X, sg, N, P) in cubes:
            um = pkg.Unmixer(S)
            hs.append(um)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat, bad = [], 0
        for um, (S, X, sg, N, P), o, ta in zip(hs, cubes, outs, arr):
            d = t0 + ta - time.perf_counter()
            if d > 0:
                time.sleep(d)
            pkg.linmin_unmix(um.h, X, N, sg, *o)
            st, _ = um.wait()
            bad += st != 0
            lat.append((time.perf_counter() - t0 - ta) * 1e3)
        end = time.perf_counter() - t0
        for um in hs:
            um.close()
        return {"value": total / end, "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99),
                "makespan_s": end, "failed": bad}

    # warm-up (first launches of each kernel size, allocator)
    served(np.zeros(n_cubes))
    res = {"workload": f"{n_cubes} cubes, N log-uniform 1e3..3e5, L in {{128,184,240}}, "
                       f"P in {{16,32,48,64}} (P-4 minerals + 4 extras), Poisson {rate:g}/s",
           "pixels": total, "unit": "pixels/s", "slots": slots, "chunk_pixels": chunk,
           "hbm_budget_gb": budget_gb, "inputs": "device-resident"}
    res["stream"] = served(arrivals)
    res["stream_plain"] = plain(arrivals)
    # a stream whose arrivals outrun the server (10x the rate): pixels/s is
    # then the server's capacity, not the arrival process
    sat_rate = 10.0 * rate
    sat = synth.poisson_arrivals(n_cubes, sat_rate)
    res["saturated_rate_per_s"] = sat_rate
    res["stream_saturated"] = served(sat)
    res["stream_saturated_plain"] = plain(sat)
    res["batch"] = served(np.zeros(n_cubes))
    # interior-point flops of the batch (each cube's own iteration counts,
    # P^3 / 3 + 6 P^2 per pixel-iteration) over its makespan
    flops = 0.0
    for (S, X, sg, N, P), o in zip(cubes, outs):
        flops += float(o[3].to(torch.float64).abs().sum().item()) * (P ** 3 / 3.0 + 6.0 * P * P)
    res["batch"]["roofline"] = {"kernel": "interior point, all cubes", "bound": "alu",
                                "achieved": flops / res["batch"]["makespan_s"] / 1e12,
                                "peak": fp32_peak, "unit": "TFLOP/s",
                                "frac": flops / res["batch"]["makespan_s"] / 1e12 / fp32_peak,
                                "note": "whole-call makespan (projection, crossover and RMS "
                                        "included): a lower bound of the solve's fraction"}
    res["batch_plain"] = plain(np.zeros(n_cubes))

    def batched():
        # linmin_unmix_batch: one queue, one interior-point launch per group
        # of cubes with the same P (a persistent grid, one work counter over
        # all their pixels); handles made beforehand, one warm-up batch
        stream = torch.cuda.Stream(device=dev)
        hs = [pkg.Unmixer(S, stream=stream) for (S, X, sg, N, P) in cubes]
        call = lambda: pkg.linmin_unmix_batch(
            [u.h for u in hs], [c[1] for c in cubes], [c[3] for c in cubes],
            [c[2] for c in cubes], [o[0] for o in outs], [o[1] for o in outs],
            [o[2] for o in outs], [o[3] for o in outs])
        call()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        call()
        bad = sum(u.wait()[0] != 0 for u in hs)
        end = time.perf_counter() - t0
        groups = len({(u.P, pkg.linmin_get_lanes(u.h)) for u in hs})
        for u in hs:
            u.close()
        fl = 0.0
        for (S, X, sg, N, P), o in zip(cubes, outs):
            fl += float(o[3].to(torch.float64).abs().sum().item()) * (P ** 3 / 3.0 + 6.0 * P * P)
        return {"value": total / end, "makespan_s": end, "failed": bad,
                "interior_point_launches": groups,
                "roofline": {"kernel": "interior point, all cubes", "bound": "alu",
                             "achieved": fl / end / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                             "frac": fl / end / 1e12 / fp32_peak}}

    res["batch_launch"] = batched()
    res["plain_note"] = ("one linmin_unmix per cube, sequential, handles created before "
                         "the timed stream")
    return res


def run_cov(pkg, dev, n_pix: int, rho: float, steps: int):
    """The same workload with band-correlated AR(1) noise unmixed under its
    full covariance (linmin_unmix_cov): pixels/s over K back-to-back calls."""
    import torch
    cube, C, Ci = synth.make_cube_cov(SPEC, rho, n_pix=n_pix or None)
    N, P = cube.N, cube.P
    stream = torch.cuda.Stream(device=dev)
    um = pkg.Unmixer(torch.from_numpy(cube.S).to(dev), stream=stream)
    X = torch.from_numpy(cube.X).to(dev)
    Cd = torch.from_numpy(Ci).to(dev)
    x = torch.empty((N, P), device=dev); sx = torch.empty((N, P), device=dev)
    rms = torch.empty((N,), device=dev); it = torch.empty((N,), dtype=torch.int32, device=dev)
    for _ in range(3):
        pkg.linmin_unmix_cov(um.h, X, N, Cd, x, sx, rms, it)
    st, nbad = um.wait()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        pkg.linmin_unmix_cov(um.h, X, N, Cd, x, sx, rms, it)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    um.close()
    return {"value": N / (ms / 1e3), "unit": "pixels/s", "ms_per_step": ms, "pixels": N,
            "noise": f"AR(1) band correlation rho = {rho}, C = D R D, D = diag(sigma)",
            "status": st, "not_converged": nbad}


def run_crism(pkg, dev, steps: int, fp32_peak: float, n_check: int = 2048):
    """The CRISM-shaped cube (640 x 480 = 307,200 pixels, L = 240, P = 48:
    44 minerals, 8 of them near-duplicates, + 4 level/slope spectra; paper
    Sec. 4.2 shape) in the exact tensor-core projection mode and the bf16
    one ("A^T y in BF16 with FP32 accumulation"): pixels/s over K
    back-to-back calls (the cube, 295 MB, is larger than L2), the
    interior-point roofline at P = 48, and the errors of the timed result
    against the oracle on a seeded sample of n_check pixels (the bf16
    error is reported, not required to meet the bar).  TF32 is not offered:
    its 10-bit inputs fail the same way bf16 does on these libraries."""
    import torch
    import oracle
    spec = synth.CRISM_307K
    cube = synth.make_cube(spec)
    N, P, L = cube.N, cube.P, cube.L
    rows = sample_rows(N, n_check)
    ref = oracle.unmix(cube.S, cube.sigma, cube.X[rows])
    X = torch.from_numpy(cube.X).to(dev)
    sg = torch.from_numpy(cube.sigma).to(dev)
    flop_per_iter = P ** 3 / 3.0 + 6.0 * P * P
    out = {"workload": spec.name, "pixels": N, "L": L, "P": P,
           "library": "44 minerals (8 near-duplicates) + 4 level/slope spectra",
           "l2": "inputs larger than L2 (cube 295 MB), no flush",
           "tf32": "not offered (10-bit inputs: same failure as bf16 on these libraries)"}
    for mode, prec in (("tc_exact", 1), ("bf16", 2)):
        stream = torch.cuda.Stream(device=dev)
        um = pkg.Unmixer(torch.from_numpy(cube.S).to(dev), stream=stream, profile=True,
                         precision=prec)
        x = torch.empty((N, P), device=dev); sx = torch.empty((N, P), device=dev)
        rms = torch.empty((N,), device=dev); it = torch.empty((N,), dtype=torch.int32, device=dev)
        for _ in range(3):
            pkg.linmin_unmix(um.h, X, N, sg, x, sx, rms, it)
        st, nbad = um.wait()
        iters = it.to(torch.float64).abs()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            pkg.linmin_unmix(um.h, X, N, sg, x, sx, rms, it)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        n_phase = min(steps, pkg.linmin.LINMIN_PHASE_RING)
        ph = {k: 0.0 for k in pkg.linmin.PHASES}
        for back in range(n_phase):
            for k, v in pkg.linmin_phase_times_at(um.h, back).items():
                ph[k] += v / n_phase
        st, nbad = um.wait()
        ipm_ms = ph["ipm"] + ph["retry"]
        achieved = float(iters.sum().item()) * flop_per_iter / (ipm_ms / 1e3) / 1e12
        acc = accuracy(cube, rows, ref, x.cpu().numpy(), sx.cpu().numpy(), rms.cpu().numpy())
        out[mode] = {"value": N / (ms / 1e3), "unit": "pixels/s", "ms_per_step": ms,
                     "phase_ms": ph, "status": st, "not_converged": nbad,
                     "mean_iters": float(iters.mean().item()),
                     "roofline": {"kernel": "ipm (interior-point launches)", "bound": "alu",
                                  "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                                  "frac": achieved / fp32_peak, "flops_per_iter": flop_per_iter},
                     "accuracy": acc}
        um.close()
    return out


def run_constraints(pkg, dev, n_pix: int, steps: int):
    """The slo (sum x <= 1) and pos (x >= 0) constraint sets on the same
    cube with the library's decreasing slope dropped (they need rank S = P,
    which the flat + two slopes break): pixels/s of each."""
    import torch
    cube = synth.make_cube(SPEC, n_pix=n_pix or None)
    keep = [j for j in range(cube.P) if j != cube.P - 2]
    S = torch.from_numpy(np.ascontiguousarray(cube.S[keep])).to(dev)
    X = torch.from_numpy(cube.X).to(dev)
    sg = torch.from_numpy(cube.sigma).to(dev)
    N, P = cube.N, len(keep)
    out = {"library": f"{P} spectra (decreasing slope dropped: rank S = P)", "pixels": N}
    for name, c in (("slo", 1), ("pos", 2)):
        stream = torch.cuda.Stream(device=dev)
        um = pkg.Unmixer(S, stream=stream, constraint=c)
        x = torch.empty((N, P), device=dev); sx = torch.empty((N, P), device=dev)
        rms = torch.empty((N,), device=dev); it = torch.empty((N,), dtype=torch.int32, device=dev)
        for _ in range(2):
            pkg.linmin_unmix(um.h, X, N, sg, x, sx, rms, it)
        st, nbad = um.wait()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            pkg.linmin_unmix(um.h, X, N, sg, x, sx, rms, it)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"value": N / (ms / 1e3), "unit": "pixels/s", "ms_per_step": ms,
                     "status": st, "not_converged": nbad,
                     "mean_iters": float(it.to(torch.float64).abs().mean().item())}
        um.close()
    return out


def run_detection(pkg, dev, cube, x, sx, rms, it, steps: int, hbm_peak: float,
                  n_second: bool = True, flush_gb: float = 4.0):
    """Detection products on the unmixed cube: eq. Threshold from the known
    truth (threshold sums kernel), then the per-pixel detection kernel with
    the three conditions of Sec. 4.  Each detection launch is timed alone
    with events on its stream, after a 4 GiB write that flushes L2 (its
    inputs, 8P + 24 bytes per pixel, fit in L2)."""
    import ctypes
    import torch
    from paper_1402_2518_gb300 import linmin
    N, P, nm = cube.N, cube.P, cube.P - 4
    stream = torch.cuda.Stream(device=dev)
    truth = torch.from_numpy(synth.truth_masks(cube.A_true, nm).view(np.int64)).to(dev)
    sums = torch.empty((ctypes.sizeof(linmin.linmin_threshold_sums),), dtype=torch.uint8,
                       device=dev)
    out = torch.empty((ctypes.sizeof(linmin.linmin_detection),), dtype=torch.uint8, device=dev)
    mask = torch.empty((N,), dtype=torch.int64, device=dev)
    # 4 GiB: flushes L2 and keeps the device busy (~0.7 ms) while the host
    # queues the timed call (pointer checks, memset, two launches), so that
    # the events bracket the kernels alone
    flush = torch.empty((int(flush_gb * (1 << 30)),), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    pkg.linmin_threshold_stats(x, truth, N, P, nm, sums, stream=stream)
    torch.cuda.synchronize()
    x_min = np.maximum(pkg.linmin_thresholds(pkg.threshold_sums(sums), nm), 0.0)
    rms_max = float(2.0 * cube.sigma.mean())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    with torch.cuda.stream(stream):
        for _ in range(3):
            pkg.linmin_detect(x, sx, rms, it, truth, N, P, nm, x_min, rms_max, mask, out,
                              stream=stream)
        for e0, e1 in ev:
            flush.fill_(1)
            e0.record(stream)
            pkg.linmin_detect(x, sx, rms, it, truth, N, P, nm, x_min, rms_max, mask, out,
                              stream=stream)
            e1.record(stream)
    torch.cuda.synchronize()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps
    t0 = time.perf_counter()
    pkg.linmin_detect(x, sx, rms, it, truth, N, P, nm, x_min, rms_max, mask, out, stream=stream)
    host_us = (time.perf_counter() - t0) * 1e6
    torch.cuda.synchronize()
    d = pkg.detection_summary(out)
    nt = int(d["n_true"][:nm].sum())
    # library auto-fit (Sec. 2.4), one call
    S = torch.from_numpy(cube.S).to(dev)
    rl = torch.empty((P, cube.L), device=dev); rn = torch.empty((P, cube.L), device=dev)
    a0 = torch.cuda.Event(enable_timing=True); a1 = torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        pkg.linmin_autofit(S, cube.L, P, rl, rn, stream=stream)
    a0.record(stream)
    pkg.linmin_autofit(S, cube.L, P, rl, rn, stream=stream)
    a1.record(stream)
    torch.cuda.synchronize()
    autofit_ms = a0.elapsed_time(a1)
    # second pass (Sec. 5): every pixel unmixed again with its detected
    # minerals and the extras (linmin_unmix_masked, K calls timed on the
    # stream like the main step)
    second = None
    if n_second:
        X = torch.from_numpy(cube.X).to(dev)
        sg = torch.from_numpy(cube.sigma).to(dev)
        um2 = pkg.Unmixer(S, stream=stream)
        x2 = torch.empty((N, P), device=dev); sx2 = torch.empty((N, P), device=dev)
        r2 = torch.empty((N,), device=dev); i2 = torch.empty((N,), dtype=torch.int32, device=dev)
        for _ in range(2):
            pkg.linmin_unmix_masked(um2.h, X, N, sg, mask, nm, x2, sx2, r2, i2)
        st2, nbad2 = um2.wait()
        b0 = torch.cuda.Event(enable_timing=True); b1 = torch.cuda.Event(enable_timing=True)
        k2 = max(3, steps // 2)
        b0.record(stream)
        for _ in range(k2):
            pkg.linmin_unmix_masked(um2.h, X, N, sg, mask, nm, x2, sx2, r2, i2)
        b1.record(stream)
        torch.cuda.synchronize()
        ms2 = b0.elapsed_time(b1) / k2
        um2.close()
        hm = mask.cpu().numpy()
        second = {"value": N / (ms2 / 1e3), "unit": "pixels/s", "ms_per_step": ms2,
                  "pixels": N, "distinct_masks": int(np.unique(hm).size), "status": st2,
                  "not_converged": nbad2,
                  "mean_iters": float(i2.to(torch.float64).abs().mean().item()),
                  "note": "linmin_unmix_masked with the detection masks of this leg"}
    byts = N * (8 * P + 24)
    gbs = byts / (ms / 1e3) / 1e9
    return {"value": N / (ms / 1e3), "unit": "pixels/s", "ms_per_call": ms,
            "host_queue_us": host_us,
            "launches_per_step": 2, "pixels": N,
            "roofline": {"kernel": "detect_kernel", "bound": "hbm", "achieved": gbs,
                         "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                         "bytes_per_pixel": 8 * P + 24, "traffic": detect_traffic(N),
                         "l2": f"{flush_gb:g} GiB write before each timed launch"},
            "thresholds": "eq. Threshold from the truth of the cube (population std)",
            "rms_max": rms_max,
            "positive_detection": int(d["true_pos"][:nm].sum()) / max(nt, 1),
            "false_detection": int(d["false_pos"][:nm].sum()) / max(N * nm - nt, 1),
            "autofit_ms": autofit_ms,
            "second_pass": second}


def main():
    global SPEC
    args = parse()
    if args.workload == "crism":
        SPEC = synth.CRISM_307K
    ws, rank, local = dist_env()
    cube = synth.make_cube(SPEC, n_pix=args.pixels or None)
    if args.impl == "reference":
        run_reference(args, cube)
        return

    import torch
    import torch.distributed as dist
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_1402_2518_gb300 as pkg
    pkg.load()
    stream = torch.cuda.Stream(device=dev)
    prec = {"df": 0, "tc": 1, "bf16": 2}[args.precision]
    um = pkg.Unmixer(torch.from_numpy(cube.S).to(dev), stream=stream, profile=True,
                     precision=prec)
    X = torch.from_numpy(cube.X).to(dev)
    sig = torch.from_numpy(cube.sigma).to(dev)
    N, P, L = cube.N, cube.P, cube.L
    x = torch.empty((N, P), device=dev)
    sx = torch.empty((N, P), device=dev)
    rms = torch.empty((N,), device=dev)
    it = torch.empty((N,), dtype=torch.int32, device=dev)
    torch.cuda.synchronize()

    def step():
        pkg.linmin_unmix(um.h, X, N, sig, x, sx, rms, it)

    for _ in range(max(args.warmup, 3)):
        step()
    st, nbad = um.wait()
    if st not in (0,):
        raise RuntimeError(f"unmix status {st}: {pkg.linmin_last_error(um.h)}")

    phase_tot = {k: 0.0 for k in pkg.linmin.PHASES}
    flops_ipm = 0.0
    iters = it.to(torch.float64).abs()
    flop_per_iter = P ** 3 / 3.0 + 6.0 * P * P
    flops_ipm = float(iters.sum().item()) * flop_per_iter
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    # phase times of the timed calls, from the library's own events on its
    # stream (it keeps the last LINMIN_PHASE_RING calls)
    n_phase = min(args.steps, pkg.linmin.LINMIN_PHASE_RING)
    for back in range(n_phase):
        for k, v in pkg.linmin_phase_times_at(um.h, back).items():
            phase_tot[k] += v * args.steps / n_phase
    launches = pkg.linmin_last_launches(um.h)
    if ws > 1:
        ms = max_over_ranks(ms, dist, dev)
        dist.barrier()
    st, nbad = um.wait()

    # end to end through the C ABI with host buffers (pinned), copies inside
    e2e_s = e2e = None
    if not args.no_e2e:
        e2e_s = run_e2e(pkg, cube, max(3, args.steps // 2), prec)
        if ws > 1:
            e2e_s = max_over_ranks(e2e_s, dist, dev)
        e2e = {"value": replicas_value(N, e2e_s, ws), "unit": "pixels/s",
               "h2d_bytes_per_step": N * L * 4 + L * 4,
               "d2h_bytes_per_step": N * (2 * P + 2) * 4}
    peak_ffma, peak_ffma2 = pkg.linmin_fp32_peak(stream)
    fp32_peak = max(peak_ffma, peak_ffma2)
    crism = None
    if not args.no_crism and rank == 0 and not args.pixels and args.workload == "omega":
        crism = run_crism(pkg, dev, max(3, args.steps // 4), fp32_peak)
    full_cov = None
    if not args.no_cov and rank == 0:
        full_cov = run_cov(pkg, dev, args.pixels, 0.5, max(3, args.steps // 4))
    constraints = None
    if not args.no_constraints and rank == 0:
        constraints = run_constraints(pkg, dev, args.pixels, max(3, args.steps // 4))
    detection = None
    if not args.no_detection and rank == 0:
        detection = run_detection(pkg, dev, cube, x, sx, rms, it, max(3, args.steps // 2),
                                  float(measured_peaks().get("hbm_gbs", 6800.0)),
                                  not args.no_second_pass, args.detect_flush_gb)
    serving = None
    if not args.no_serving and rank == 0:
        serving = run_serving(pkg, dev, args.serving_cubes, args.serving_rate,
                              args.serving_budget_gb, args.serving_slots, args.serving_chunk, fp32_peak)
    if rank != 0:
        dist.barrier() if ws > 1 else None
        return

    value = replicas_value(N, ms / 1e3, ws)
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    nsm = props.multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_derived = nsm * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12   # TFLOP/s
    ipm_ms = (phase_tot["ipm"] + phase_tot["retry"]) / args.steps
    achieved = flops_ipm / (ipm_ms / 1e3) / 1e12
    clocks = clk.summary()
    # accuracy of the timed call's result: against the CPU baseline's own
    # oracle run on its prefix, else on a seeded sample the oracle recomputes
    xh, sxh, rmsh = x.cpu().numpy(), sx.cpu().numpy(), rms.cpu().numpy()
    if args.no_cpu_baseline:
        import oracle
        cpu = None
        rows = sample_rows(N, args.check_pixels)
        ref = oracle.unmix(cube.S, cube.sigma, cube.X[rows])
    else:
        cpu, rows, ref = cpu_baseline(cube, args.cpu_seconds)
    acc = accuracy(cube, rows, ref, xh, sxh, rmsh)
    if not acc["max_abs_err"] <= X_TOL:
        raise SystemExit(f"timed result misses the bar: max |x - x_oracle| = "
                         f"{acc['max_abs_err']:.3e} > {X_TOL:g} on {acc['pixels']} pixels")
    line = {
        "metric": METRIC, "value": value, "unit": "pixels/s", "n_gpus": ws,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"df": "f32 (double-float projection and crossover)",
                  "tc": "f32 (bf16 tensor-core projection on exact 8-bit slices, "
                        "double-float crossover)",
                  "bf16": "f32 (bf16 tensor-core projection, double-float crossover)"}[args.precision],
        "data": "synthetic",
        "config": {"workload": SPEC.name, "pixels": N, "L": L, "P": P,
                   "library": (f"{SPEC.n_minerals} minerals"
                               + (f" ({SPEC.n_near_dup} near-duplicates)" if SPEC.n_near_dup else "")
                               + f" + {SPEC.n_extras} level/slope spectra"),
                   "l2": (f"inputs larger than L2 (cube {N * L * 4 / 1e6:.0f} MB), no flush"
                          if N * L * 4 > 129e6 else "cube smaller than L2 (a reduced run)"),
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"kernel": "ipm (interior-point launches: all pixels + retry list)",
                     "bound": "alu", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": ipm_traffic(N) if args.workload == "omega" else None,
                     "traffic_note": "DRAM bytes of the main IPM launch (ncu on 65,536 "
                                     "pixels, scaled by pixel count)",
                     "peak_note": (f"measured by linmin_fp32_peak in this run: FFMA "
                                   f"{peak_ffma:.2f}, FFMA2 {peak_ffma2:.2f} TFLOP/s (the larger); "
                                   f"derived {fp32_derived:.2f} = {nsm} SMs x 128 lanes x 2 x "
                                   f"{max_mhz:.0f} MHz"),
                     "peak_derived": fp32_derived,
                     "window_note": "time = the ipm and retry phases; retry also holds the "
                                    "retry list's support, sort and crossover launches, so "
                                    "the fraction is slightly conservative",
                     "flops_per_iter": flop_per_iter,
                     "mean_iters": float(iters.mean().item())},
        "projection": projection_roofline(N, L, P, phase_tot["project"] / args.steps,
                                          float(peaks.get("hbm_gbs", 6800.0))),
        "accuracy": acc,
        "phase_ms": {k: v / args.steps for k, v in phase_tot.items()},
        "not_converged": nbad,
        "e2e": e2e,
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "serving": serving,
        "crism": crism,
        "full_covariance": full_cov,
        "constraints": constraints,
        "detection": detection,
    }
    print(json.dumps(line))
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    um.close()


if __name__ == "__main__":
    main()

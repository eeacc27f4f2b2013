#!/usr/bin/env python
"""Throughput of the NUFFT kernel smoother on one GB300 (or N replicas).

One step = the whole hot path on the 2-D local-linear workload
(N = 10^6 samples from a clipped 3-Gaussian mixture, 256 x 256 grid,
H = diag(0.01^2, 0.015^2), FP32 with FP64 solves, tol 1e-6):
  bin + stable sort of the samples (fkreg_set_points),
  fkreg_df with y and 10 on-device Gaussian probes (Table 1 default Np):
    type-1 spreading of 12 strengths, FFT, kernel multiply + deconvolution,
    inverse FFT, FP64 grid solves (6 moment + 3 response grids -> mhat, mask),
    type-2 interpolation of 39 fields at every sample with the FP64
    at-sample solve, RSS, Monte-Carlo DF, exact trace and GCV,
  fkreg_variance: spreading + smoothing of the squared residuals (eq. 23).
value = N * (1 response + 10 probes + 1 variance response) * bandwidths / step time,
in sample-points per second, summed over all ranks (independent replicas).

--impl reference times the FP64 oracle (direct sums) on the host cores on a
bounded sample of the same step and extrapolates per query point.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_PROBES = 10
WORKLOAD = "ll2d-1M-256sq-LL-f32-tol1e-6"
METRIC = "sample-pts/sec of NUFFT smoothing at rel err<=1e-5 vs plain FP64; % HBM roofline"
UNIT = "sample-pts/s"
DTYPE_F32 = "f32 fields, f64 grid solves, compensated-f32 sample solves"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other configurations after the headline line's measurement")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", default="ll2d",
                    choices=["ll2d", "ll2d_sort", "nw1d", "nw3d_df", "ll2d_gcv", "uneven",
                             "ll2d_plain64", "ll2d_plain32", "ll2d_logvar", "ll2d_epan"],
                    help="ll2d is the headline line; the others measure the remaining "
                         "configurations (1-D NW FP64, 3-D NW + DF sweep, 2-D LL GCV "
                         "forward + backward, 64 uneven problems in one graph) and the "
                         "plain single-response form of the ll2d step (FP64 or FP32: "
                         "one smooth call per response / probe, no stacking), and the "
                         "ll2d smooth followed by the log-variance estimator (eqs. 24-26), "
                         "and the ll2d step with the Epanechnikov kernel (direct sums)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="sample-count multiplier for the extra workloads (1 = full size)")
    return ap.parse_args()


def hbm_peak():
    """HBM peak: the measured STREAM-style copy bandwidth in MEASURED_PEAKS.json."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons around a region.

    The sampler is running (its first line written) before the region
    starts; the samples stamped inside the region, widened by one sampling
    interval on each side, are kept.  A region shorter than the interval
    may hold none: the sample nearest to it then stands in, and
    ``in_region`` says which case it was.
    """

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, interval_ms: int = 20):
        self.index = index
        self.iv = interval_ms / 1e3
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms",
                                       str(int(self.iv * 1e3))],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
            return
        t = time.time()
        while time.time() - t < 5.0 and self.p.poll() is None:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.005)
        self.t0 = time.time()

    @staticmethod
    def _stamp(text: str):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(text, fmt).timestamp()
            except ValueError:
                pass
        return None

    def stop(self):
        self.t1 = time.time()
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(2 * self.iv)   # the sample just after the region
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                sm, smax = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            active = {nm for nm, v in zip(names, parts[6:10]) if v.lower() == "active"}
            rows.append((self._stamp(parts[0]), sm, smax, active))
        os.unlink(self.f.name)
        t0 = self.t0 if self.t0 is not None else self.t1
        inside = [r for r in rows
                  if r[0] is not None and t0 - self.iv <= r[0] <= self.t1 + self.iv]
        keep = inside
        if not keep:
            stamped = [r for r in rows if r[0] is not None]
            mid = 0.5 * (t0 + self.t1)
            keep = [min(stamped, key=lambda r: abs(r[0] - mid))] if stamped else rows
        reasons = set()
        for r in keep:
            reasons |= r[3]
        return {"sm_mhz": statistics.median(r[1] for r in keep) if keep else None,
                "sm_max_mhz": max(r[2] for r in keep) if keep else None,
                "reasons": sorted(reasons), "samples": len(keep), "in_region": bool(inside),
                "interval_ms": int(self.iv * 1e3), "region_ms": round((self.t1 - t0) * 1e3, 1)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# DRAM bytes (read + write) per launch of the dominant kernels, from one ncu
# capture of the bench command (see profiles/); None where the kernel changed
# after the counters were taken.
TRAFFIC = {"interp": 79684864, "spread": 62001920}


def max_over_ranks(ms: float, world: int, device) -> float:
    """The job's time: the slowest rank's (all-reduce MAX over the ranks)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_step: float, steps: int, world: int, total_ms: float) -> float:
    """Units all ranks processed (each rank runs one replica) per second of the job."""
    return world * units_per_step * steps / (total_ms / 1e3)


def algorithmic(plan, n, n_probes):
    """Algorithmic bytes / flops per launch of the spreading and interpolation kernels."""
    T = 4
    d = plan.d
    S = 1 + plan.n_rhs + n_probes
    nf = int(math.prod(plan.geom["nf"]))
    w = plan.geom["w"]
    # spread: read d coordinates + S strengths per sample, write S fine grids once
    spread_bytes = n * (d * T + S * T) + S * nf * T
    spread_flops = 2 * n * S * w ** d
    F2 = plan.ns + (plan.n_rhs + n_probes) * plan.nt
    # interp: read coordinates, permutation, responses/probes; read the F2 fine
    # grids once; write mhat at the samples
    interp_bytes = n * (d * T + 4 + (plan.n_rhs + n_probes) * T + plan.n_rhs * T) + F2 * nf * T
    interp_flops = 2 * n * F2 * w ** d
    return {"spread": (spread_bytes, spread_flops), "interp": (interp_bytes, interp_flops)}


STEP_WANT = ("mhat_grid", "mask", "mhat_at_x")


def ll2d_plan(w, device):
    """The plan of the headline step (2-D local linear, FP32, y + N_PROBES probes)."""
    from paper_2204_07716_gb300 import fkreg
    return fkreg.Plan(2, 1, w.grid_n, w.lo, w.hi, w.H, max_n=w.n, n_rhs=1, max_probes=N_PROBES,
                      tol=w.tol, precision="f32", device=device)


def ll2d_step(plan, x, y, seed):
    """One headline step: bin sort, df with y and N_PROBES device probes, variance pass."""
    plan.set_points(x)
    out = plan.df(y, N_PROBES, seed=seed, want=STEP_WANT)
    s2 = plan.variance(y, out["mhat_at_x"])
    return out, s2


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2204_07716_gb300 import build as fkbuild
    from paper_2204_07716_gb300 import fkreg, inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        fkbuild.build()
    if world > 1:
        dist.barrier()
    w = inputs.ll2d()
    n = w.n
    plan = ll2d_plan(w, dev)
    x = torch.tensor(w.x, dtype=torch.float32, device=dev)
    y = torch.tensor(w.y, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(k, xx, yy):
        return ll2d_step(plan, xx, yy, 1000 + k)

    for k in range(args.warmup):
        step(k, x, y)
    plan.sync()
    # the whole step (sort, df with device probes, variance) as one CUDA
    # graph: every kernel, copy and FFT of the eager step, one launch
    graph = fkreg.StepGraph(lambda: step(0, x, y))
    for _ in range(args.warmup):
        graph.replay()
    clocks = Clocks(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    for k in range(args.steps):
        flush.fill_(float(k))                 # evict L2 between steps (512 MB > 129 MB)
        ev[k][0].record(stream)
        graph.replay()
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    plan.sync()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # per-stage launch times and kernel counts: the same steps issued eagerly
    # with the library's stage events on
    plan.stage_times()                      # reset timers and launch counter
    plan.set_timing(True)
    for k in range(args.steps):
        flush.fill_(float(k))
        step(args.warmup + k, x, y)
    torch.cuda.synchronize(dev)
    plan.sync()
    stage_ms, stage_calls, launches = plan.stage_times()
    plan.set_timing(False)
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    units_per_step = n * (1 + N_PROBES + 1) * plan.n_bw
    value = whole_job_value(units_per_step, args.steps, world, total_ms)

    # e2e: host pinned inputs, copies inside the timed region, results read
    # back.  Two input buffers, each with its own captured graph, let the next
    # step's host-to-device copy (a stream of its own) run under the current
    # step's kernels; each step's interval runs from its graph's start (the
    # first step: from its copy) to the end of its results' device-to-host
    # copy, so nothing that is not hidden under a timed graph goes unmeasured.
    xh = torch.tensor(w.x, dtype=torch.float32).pin_memory()
    yh = torch.tensor(w.y, dtype=torch.float32).pin_memory()
    x2 = torch.empty_like(x)
    y2 = torch.empty_like(y)
    x2.copy_(x)
    y2.copy_(y)
    graph2 = fkreg.StepGraph(lambda: step(0, x2, y2))
    bufs = [(x, y, graph), (x2, y2, graph2)]
    hosts = [(torch.empty((plan.n_bw, 1) + w.grid_n, dtype=torch.float32).pin_memory(),
              torch.empty((plan.n_bw, 1), dtype=torch.float64).pin_memory(),
              torch.empty((plan.n_bw, 1) + w.grid_n, dtype=torch.float32).pin_memory())
             for _ in range(2)]
    h2d_stream, d2h_stream = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]

    def h2d_into(j):
        h2d_stream.wait_stream(stream)        # after the flush and the graph that used buffer j
        with torch.cuda.stream(h2d_stream):
            bufs[j][0].copy_(xh, non_blocking=True)
            bufs[j][1].copy_(yh, non_blocking=True)
            ev_in[j].record(h2d_stream)

    torch.cuda.synchronize(dev)
    e2e_ev[0][0].record(stream)
    h2d_into(0)
    for k in range(args.steps):
        i = k % 2
        if k > 0:
            flush.fill_(float(k))             # between timed steps, outside the intervals
            e2e_ev[k][0].record(stream)
        if k + 1 < args.steps:
            h2d_into((k + 1) % 2)             # the next step's inputs, under this step's kernels
        stream.wait_event(ev_in[i])
        bufs[i][2].replay()
        ev_done[i].record(stream)
        d2h_stream.wait_event(ev_done[i])
        gout, gs2 = bufs[i][2].outputs
        with torch.cuda.stream(d2h_stream):
            hosts[i][0].copy_(gout["mhat_grid"], non_blocking=True)
            hosts[i][1].copy_(gout["gcv"], non_blocking=True)
            hosts[i][2].copy_(gs2, non_blocking=True)
            ev_out[i].record(d2h_stream)
        stream.wait_event(ev_out[i])
        e2e_ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    plan.sync()
    mh_host, gcv_host, s2_host = hosts[0]
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in e2e_ev), world, dev)
    e2e_value = whole_job_value(units_per_step, args.steps, world, e2e_ms)
    h2d = xh.numel() * 4 + yh.numel() * 4
    d2h = mh_host.numel() * 4 + gcv_host.numel() * 8 + s2_host.numel() * 4

    # roofline of the dominant kernel stage.  The spreading and interpolation
    # kernels do w^d multiply-adds per sample and field against a few bytes of
    # HBM traffic: the FP32 FMA rate is their roofline (bound "alu"); the HBM
    # figure of the same launch is reported beside it.
    own = {k: v for k, v in stage_ms.items() if k not in ("fft_fwd", "fft_grid", "fft_t2")}
    dom = max(own, key=own.get)
    hbm, hbm_kind = hbm_peak()
    # the SM-side peaks measured on this GPU in this run (after the timed region)
    sm = fkreg.measure_peaks(dev)
    fp32_peak = max(sm["fp32_tflops"], sm["fp32x2_tflops"])
    alg = algorithmic(plan, n, N_PROBES)
    roof = None
    if dom in alg and stage_calls[dom]:
        # the interp stage is one launch per bandwidth; the spread stage holds
        # the df launches (1 + R + probes strengths) and the variance launch
        per_launch_ms = stage_ms[dom] / stage_calls[dom]
        bytes_per_launch, flops_per_launch = alg[dom]
        achieved = flops_per_launch / (per_launch_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": round(achieved, 2),
                "peak": round(fp32_peak, 1), "unit": "TFLOP/s",
                "frac": round(achieved / fp32_peak, 4),
                "traffic": TRAFFIC.get(dom),
                "peak_source": "measured in this run: FP32 FMA microbenchmark (fkreg_measure_peaks)",
                "launch_ms": round(per_launch_ms, 4),
                "hbm_achieved_gbs": round(bytes_per_launch / (per_launch_ms / 1e3) / 1e9, 1),
                "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_kind}
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_F32, "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "grid": list(w.grid_n), "order": 1,
                   "bandwidth_sd": [0.01, 0.015], "probes": N_PROBES, "tol": w.tol,
                   "units_per_step": units_per_step, "l2": "flushed (512 MB write) between steps",
                   "graph": "whole step captured once; one CUDA graph replay per step",
                   "parallelism": f"replicas{world}"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms / args.steps,
                "copies": "pinned host buffers; two input buffers, the next step's "
                          "host-to-device copy under the current step's kernels"},
        "gpu_launches": int(launches),   # eager steps = graph replays: same kernels
        "roofline": roof,
        "stages_ms_per_step": {k: round(v / args.steps, 4) for k, v in stage_ms.items()},
        "sm_peaks": {k: (round(v, 2) if isinstance(v, float) else
                         ([round(u, 2) for u in v] if isinstance(v, list) else v))
                     for k, v in sm.items()},
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_extra:
        # the other configurations and the plain single-response FP64 form of
        # this step, each timed on its own (device events, L2 flushed)
        plan.close()
        del graph, graph2, bufs
        torch.cuda.empty_cache()
        cfgs = {}
        for wl, st, wu in EXTRA_RUNS:
            try:
                r = measure_workload(wl, st, wu, 1.0, dev)
                cfgs[wl] = {k: r[k] for k in ("ms_per_step", "value", "unit", "dtype", "config",
                                              "steps", "warmup", "latency_ms", "clocks",
                                              "stages_ms_per_step", "roofline") if k in r}
            except Exception as e:          # reported, not hidden: the line still prints
                cfgs[wl] = {"error": f"{type(e).__name__}: {e}"[:300]}
        result["configs"] = cfgs
        p64 = cfgs.get("ll2d_plain64", {})
        if "ms_per_step" in p64:
            result["plain_f64_ms_per_step"] = p64["ms_per_step"]
            result["batched_vs_plain"] = p64["ms_per_step"] / result["ms_per_step"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


def oracle_step_estimate(w, seconds: float):
    """Time the FP64 oracle on a bounded sample of one bench step, extrapolate.

    The oracle's cost per query point is O(N): a grid point needs the 6 s-sums
    and 3 t-sums of y (grid pass) plus 3 t-sums of the residuals (variance
    pass); a sample point needs 6 s-sums and 3 t-sums for y and each probe.
    The sample evaluates a few grid and sample points and scales by M and N.
    """
    import numpy as np

    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    gp = oracle.grid_points(w.grid_n, w.lo, w.hi)
    x = w.x.astype(np.float32).astype(np.float64)
    y = w.y.astype(np.float32).astype(np.float64)
    z = oracle.probes(7, N_PROBES, w.n)
    rng = np.random.default_rng(0)
    # calibrate with a tiny sample, then size the timed sample to ~seconds
    def run(qg, qs):
        t0 = time.perf_counter()
        gi = rng.choice(gp.shape[0], size=qg, replace=False)
        oracle.smooth_at(x, np.concatenate([y, y]), w.H[0], 1, gp[gi], nthreads=cores)
        si = rng.choice(w.n, size=qs, replace=False)
        oracle.smooth_at(x, np.concatenate([y, z]), w.H[0], 1, x[si], nthreads=cores)
        return time.perf_counter() - t0

    tg = run(cores, 0) / cores
    ts = run(0, cores) / cores
    qg = max(cores, int(0.4 * seconds / max(tg, 1e-9)))
    qs = max(cores, int(0.6 * seconds / max(ts, 1e-9)))
    t = run(qg, 0)
    tg = t / qg
    t2 = run(0, qs)
    ts = t2 / qs
    M = gp.shape[0]
    full_s = tg * M + ts * w.n
    units = w.n * (1 + N_PROBES + 1)
    return {"value": units / full_s, "full_step_s": full_s, "cores": cores,
            "sample": f"{qg} grid points + {qs} sample points of the step (direct FP64 sums "
                      f"over all {w.n} samples each), extrapolated to {M} grid points and "
                      f"{w.n} sample points",
            "sample_s": t + t2}


def cpu_baseline(w, seconds):
    r = oracle_step_estimate(w, seconds)
    return {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
            "sample": r["sample"], "extrapolated_full_step_s": r["full_step_s"]}


def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_2204_07716_gb300 import inputs

    w = inputs.ll2d()
    per_step = max(2.0, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_step_estimate(w, per_step)
    vals, secs = [], []
    for _ in range(args.steps):
        r = oracle_step_estimate(w, per_step)
        vals.append(r["value"])
        secs.append(r["full_step_s"])
    value = statistics.median(vals)
    ms = statistics.median(secs) * 1e3
    cores = os.cpu_count() or 1
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": w.n, "grid": list(w.grid_n), "order": 1,
                   "probes": N_PROBES, "parallelism": "host cores"},
        "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT,
                         "sample": r["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_extra(args):
    """Timed steps of one of the other configurations (one GPU, device events)."""
    import torch

    from paper_2204_07716_gb300 import build as fkbuild

    fkbuild.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    res = measure_workload(args.workload, args.steps, args.warmup, args.scale, dev)
    print(json.dumps(res), flush=True)


# The other configurations, timed after the headline in the default run: a
# few steps each (the 3-D sweep's step is about 0.7 s), so the whole run ends
# within minutes.
EXTRA_RUNS = (("ll2d_plain64", 5, 3), ("nw1d", 20, 3), ("nw3d_df", 3, 3), ("ll2d_gcv", 10, 3),
              ("uneven", 10, 3), ("ll2d_epan", 5, 3), ("ll2d_logvar", 10, 3))


def sweep_roofline(plan, w, n_probes, st_ms, st_calls, dev):
    """Roofline of the dominant own stage of the 3-D sweep: the spreading
    (N w^d strengths multiply-adds per launch) or the interpolation (N w^d
    fields multiply-adds per launch, one launch per bandwidth), against the
    FP32 FMA rate measured on this GPU."""
    from paper_2204_07716_gb300 import fkreg
    own = {k: v for k, v in st_ms.items() if k in ("spread", "interp") and st_calls[k]}
    if not own:
        return None
    dom = max(own, key=own.get)
    wd = plan.geom["w"] ** w.d
    per_sample = (1 + w.y.shape[0] + n_probes) if dom == "spread" else \
        (plan.ns + (w.y.shape[0] + n_probes) * plan.nt)
    flops = 2.0 * w.n * wd * per_sample
    per_launch_ms = st_ms[dom] / st_calls[dom]
    sm = fkreg.measure_peaks(dev)
    peak = max(sm["fp32_tflops"], sm["fp32x2_tflops"])
    achieved = flops / (per_launch_ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": dom, "achieved": round(achieved, 2), "peak": round(peak, 1),
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
            "peak_source": "measured in this run: FP32 FMA microbenchmark (fkreg_measure_peaks)",
            "launch_ms": round(per_launch_ms, 3), "launches_per_step": int(st_calls[dom]),
            "algorithmic_flops_per_launch": flops}


def measure_workload(wl, steps, warmup, sc, dev):
    """Timed steps of configuration wl on device dev; returns the result line."""
    import numpy as np
    import torch

    from paper_2204_07716_gb300 import fkreg, inputs

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    extra = {}
    if wl == "uneven":
        ws = inputs.uneven(scale=sc)
        probs = [dict(d=w.d, order=1, grid_n=w.grid_n, lo=w.lo, hi=w.hi, H=w.H, max_n=w.n,
                      tol=w.tol, precision="f32", y_complex=True) for w in ws]
        xs = [torch.tensor(w.x, dtype=torch.float32, device=dev) for w in ws]
        ys = [torch.view_as_real(torch.tensor(w.y[0], dtype=torch.complex64, device=dev)).contiguous()
              for w in ws]
        batch = fkreg.Batch(probs, device=dev)
        batch.capture(xs, ys, variance=True)
        step = lambda k: batch.launch()
        units = sum(w.n for w in ws) * 2
        cfg = {"workload": f"uneven-{len(ws)}problems-complex-LL+variance",
               "n_total": sum(w.n for w in ws), "problems": len(ws),
               "dims": [w.d for w in ws].count(2), "graph": "one captured CUDA graph"}
        dtype = DTYPE_F32
    elif wl == "ll2d_sort":
        # the bin sort of the headline step alone (fkreg_set_points)
        w = inputs.ll2d(n=int(1_000_000 * sc))
        plan = fkreg.Plan(w.d, w.order, w.grid_n, w.lo, w.hi, w.H, max_n=w.n, n_rhs=1,
                          max_probes=10, tol=w.tol, precision="f32", device=dev)
        x = torch.tensor(w.x, dtype=torch.float32, device=dev)

        def step(k):
            plan.set_points(x)
        units = w.n
        cfg = {"workload": "ll2d-1M-256sq-bin-sort", "n": w.n, "geometry": plan.geom}
        dtype = "u32 keys"
        extra["plan"] = plan
    elif wl == "ll2d_epan":
        # the headline step (df with y + 10 probes, then the variance pass)
        # with the compact Epanechnikov kernel: direct sums, no NUFFT
        w = inputs.ll2d(n=int(1_000_000 * sc))
        np_ = 10
        plan = fkreg.Plan(w.d, w.order, w.grid_n, w.lo, w.hi, w.H, max_n=w.n, n_rhs=1,
                          max_probes=np_, tol=w.tol, precision="f32", device=dev,
                          kernel="epanechnikov")
        x = torch.tensor(w.x, dtype=torch.float32, device=dev)
        y = torch.tensor(w.y[0], dtype=torch.float32, device=dev)

        def step(k):
            plan.set_points(x)
            o = plan.df(y, np_, seed=k, want=("mhat_grid", "mask", "mhat_at_x"))
            plan.variance(y, o["mhat_at_x"])
        units = w.n * (1 + np_ + 1)
        cfg = {"workload": "ll2d-1M-256sq-LL-epanechnikov-direct-f32", "n": w.n,
               "grid": list(w.grid_n), "probes": np_, "geometry": plan.geom}
        dtype = DTYPE_F32
        extra["plan"] = plan
    elif wl == "ll2d_logvar":
        # smooth y, then the log-variance estimator on its residuals
        w = inputs.ll2d(n=int(1_000_000 * sc))
        plan = fkreg.Plan(w.d, w.order, w.grid_n, w.lo, w.hi, w.H, max_n=w.n, n_rhs=1,
                          tol=w.tol, precision="f32", device=dev)
        x = torch.tensor(w.x, dtype=torch.float32, device=dev)
        y = torch.tensor(w.y[0], dtype=torch.float32, device=dev)

        def step(k):
            plan.set_points(x)
            o = plan.smooth(y, want=("mhat_grid", "mask", "mhat_at_x"))
            plan.log_variance(y, o["mhat_at_x"])
        units = w.n * 2
        cfg = {"workload": "ll2d-1M-256sq-LL-smooth+logvariance-f32-tol1e-6", "n": w.n,
               "grid": list(w.grid_n), "geometry": plan.geom}
        dtype = DTYPE_F32
        extra["plan"] = plan
    elif wl in ("ll2d_plain64", "ll2d_plain32"):
        # the ll2d step without stacking: y and each of the 10 probes is its
        # own smooth call (one response per launch chain), then the variance
        prec = "f64" if wl == "ll2d_plain64" else "f32"
        w = inputs.ll2d(n=int(1_000_000 * sc))
        np_ = 10
        dt = torch.float32 if prec == "f32" else torch.float64
        plan = fkreg.Plan(w.d, w.order, w.grid_n, w.lo, w.hi, w.H, max_n=w.n, n_rhs=1,
                          tol=w.tol, precision=prec, device=dev)
        x = torch.tensor(w.x, dtype=dt, device=dev)
        ys = [torch.tensor(w.y[0], dtype=dt, device=dev)] + \
             [torch.tensor(z, dtype=dt, device=dev)
              for z in inputs.gaussian_probes(np_, w.n, inputs.SEED_BASE + 99)]

        def step(k):
            plan.set_points(x)
            outs = [plan.smooth(yr, want=("mhat_grid", "mask", "mhat_at_x")) for yr in ys]
            plan.variance(ys[0], outs[0]["mhat_at_x"])
        units = w.n * (1 + np_ + 1)
        cfg = {"workload": f"ll2d-1M-256sq-LL-plain-{prec}-1rhs-per-call-tol1e-6",
               "n": w.n, "grid": list(w.grid_n), "responses_per_call": 1,
               "calls_per_step": 1 + np_, "geometry": plan.geom}
        dtype = "f64" if prec == "f64" else DTYPE_F32
        extra["plan"] = plan
    else:
        if wl == "nw1d":
            w = inputs.nw1d(n=int(10_000 * sc))
            np_ = 0
        elif wl == "nw3d_df":
            w = inputs.nw3d_df(n=int(4_000_000 * sc))
            np_ = w.n_probes
        else:
            w = inputs.ll2d_gcv(n=int(2_000_000 * sc))
            np_ = w.n_probes
        flags = fkreg.FKREG_WANT_BACKWARD if wl == "ll2d_gcv" else 0
        if wl == "nw3d_df":
            # the bandwidth sweep with a Fourier period per group of bandwidths
            plan = fkreg.Sweep(w.d, w.order, w.grid_n, w.lo, w.hi, w.H, max_n=w.n,
                               max_probes=np_, tol=w.tol, precision=w.precision, device=dev,
                               max_groups=2)
        else:
            plan = fkreg.Plan(w.d, w.order, w.grid_n, w.lo, w.hi, w.H, max_n=w.n,
                              max_probes=np_, tol=w.tol, precision=w.precision, flags=flags,
                              device=dev)
        dt = torch.float32 if w.precision == "f32" else torch.float64
        x = torch.tensor(w.x, dtype=dt, device=dev)
        y = torch.tensor(w.y, dtype=dt, device=dev)
        if wl == "nw1d":
            def step(k):
                plan.set_points(x)
                plan.smooth(y, want=("mhat_grid", "mask"))
            units = w.n
        elif wl == "nw3d_df":
            def step(k):
                plan.set_points(x)
                plan.df(y, np_, seed=k, want=("mhat_grid", "mask"))
            units = w.n * (1 + np_) * w.n_bw
        else:
            def step(k):
                plan.set_points(x)
                plan.backward(y[0], np_, seed=k)
            units = w.n * (1 + np_)
        cfg = {"workload": {"nw1d": "nw1d-10k-256-NW-f64-tol1e-9",
                            "nw3d_df": "nw3d-4M-64cube-NW-16bw-32probes-f32-tol1e-6",
                            "ll2d_gcv": "ll2d-2M-512sq-LL-GCV-fwd+bwd-f32-tol1e-6"}[wl],
               "n": w.n, "grid": list(w.grid_n), "bandwidths": w.n_bw, "probes": np_,
               "geometry": plan.geom}
        if wl == "nw3d_df":
            first, geoms = plan.groups()
            cfg["period_groups"] = [{"bandwidths": [first[i], first[i + 1]],
                                     "period": geoms[i]["period"][0], "nf": geoms[i]["nf"][0]}
                                    for i in range(len(first) - 1)]
        dtype = "f64" if w.precision == "f64" else DTYPE_F32
        extra["plan"] = plan
    for k in range(warmup):
        step(k)
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    clocks = Clocks(0)
    clocks.start()
    stream = torch.cuda.current_stream(dev)
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        step(warmup + k)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    res = {"metric": METRIC, "value": units * steps / (sum(ms) / 1e3), "unit": UNIT,
           "n_gpus": 1, "steps": steps, "warmup": warmup,
           "ms_per_step": sum(ms) / steps, "ms_step_median": float(np.median(ms)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
           "data": "synthetic", "config": cfg, "clocks": clk}
    if wl == "uneven":
        lat = batch.latencies()
        res["latency_ms"] = {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                             "max": float(lat.max())}
        iso = []
        for i, p in enumerate(probs):        # isolated per-problem latency (one plan, same inputs)
            if i % 8:
                continue
            pl = fkreg.Plan(**p, device=dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            pl.set_points(xs[i])
            o = pl.smooth(ys[i], want=("mhat_grid", "mask", "mhat_at_x"))
            pl.variance(ys[i], o["mhat_at_x"])
            e0.record()
            pl.set_points(xs[i])
            o = pl.smooth(ys[i], want=("mhat_grid", "mask", "mhat_at_x"))
            pl.variance(ys[i], o["mhat_at_x"])
            e1.record()
            e1.synchronize()
            iso.append(e0.elapsed_time(e1))
            pl.close()
        res["isolated_latency_ms_sampled"] = {"p50": float(np.percentile(iso, 50)),
                                              "max": float(max(iso)), "count": len(iso)}
    else:
        plan = extra["plan"]
        plan.stage_times()          # drop the counts of the timed steps
        plan.set_timing(True)
        step(0)
        torch.cuda.synchronize(dev)
        st_ms, st_calls, launches = plan.stage_times()
        plan.set_timing(False)
        res["stages_ms_per_step"] = {k: round(v, 4) for k, v in st_ms.items()}
        res["gpu_launches_per_step"] = launches
        if wl == "nw3d_df":
            res["roofline"] = sweep_roofline(plan, w, np_, st_ms, st_calls, dev)
    for v in list(extra.values()) + ([batch] if wl == "uneven" else []):
        v.close()
    del flush
    torch.cuda.empty_cache()
    return res


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload != "ll2d":
        if rank == 0:
            run_extra(args)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()

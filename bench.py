"""Benchmark: reciprocal averaged-intensity evaluations per second on one GB300.

One step = one cold reciprocal evaluation of the 200-lambda collimator workload
(500 cells, nx = 4040, ny = 160, 646k unknowns, annular light 10-30 deg, output angle
0): new pillar widths -> raster + assembly -> block-cyclic-reduction factorisation ->
reciprocal solve with FP64 stencil refinement -> FP64 Toeplitz quadratic form (every
row of the hot path except the brute-force comparison, which is timed separately on
the same factorisation and reported under "bruteforce").

Timed on the device with CUDA events on the library's stream, after W warm-up steps,
bracketed by a barrier and synchronisation; the factor store (1.2 GB in FP32, 2.5 GB in
FP64) is far larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp32|fp64]
  python bench.py --impl reference ...   (the FP64 CPU oracle, time-boxed)

Multi-GPU (torchrun): replicas only -- each rank evaluates its own designs; value is
the total over ranks divided by the slowest rank's time ("scaling": "weak").
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
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "reciprocal avg-intensity evals/s at 200λ (FP32+refine vs FP64), p50/p99 ms"
WORKLOAD = "c2_collimator"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
FP64_NOMINAL_TFLOPS = 1.25


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, ws: int) -> float:
    """The largest x over the ranks (the slowest rank's time sets a replica run's value)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _replica_seeds(rank: int, n: int) -> list:
    """Design seeds of one replica: disjoint across ranks, so every rank evaluates its own
    designs (replicas only: no data is exchanged between ranks)."""
    return [rank * 1_000_000 + s for s in range(n)]


def _replica_value(ws: int, steps: int, slowest_ms: float) -> float:
    """Whole-job evaluations per second: all ranks' evaluations over the slowest rank's time."""
    return ws * steps / (slowest_ms * 1e-3)


# DRAM bytes (read + write) per ny x ny block inverted by the FP32 tensor-core Gauss-Jordan
# kernel, from one ncu capture of its 1010-block launch in the 200-wavelength factorisation
# (225.6 MB read + 155.2 MB written; algorithmic 409.6 KB per block).  Only valid for ny = 160
# and that kernel as it stands.
GJ_TC_DRAM_BYTES_PER_BLOCK_NY160 = (225.58208e6 + 155.15264e6) / 1010
# nominal dense TF32 / BF16 tensor rate (1.1 / 2.25 PFLOP/s)
TF32_OVER_BF16 = 1.1 / 2.25


def _roofline(fam: str, stats: dict, prec: int, peaks: dict, peak_kind: str, ny: int = 0,
              live: dict | None = None):
    """Roofline record for one kernel family from the library's profiler totals.

    live: the arithmetic peaks measured in this run (rci_measure_peaks: FP32 FFMA, FP64
    DFMA, tcgen05 TF32, ...); without them the FP32 rate is derived from unit counts and
    clock, FP64 is nominal and TF32 a nominal ratio of the bf16 peak file."""
    ms = stats["ms"]
    if ms <= 0:
        return None
    if fam == "gemm" and prec != 0:
        # 3xTF32 complex GEMMs on tcgen05: three tensor products per complex product, each
        # the 4 real products of the complex multiply -> 3x the algorithmic complex flops
        tflops = 3.0 * stats["flops"] / (ms * 1e-3) / 1e12
        if live and live.get("tf32_tcgen05_tflops"):
            peak = live["tf32_tcgen05_tflops"]
            src = "measured in this run: tcgen05.mma kind::tf32 128x256 loop on every SM"
        else:
            peak = peaks.get("bf16_tflops_sustained", 1700.0) * TF32_OVER_BF16
            src = f"{peak_kind} sustained bf16 x 1.1/2.25 (TF32)"
        return {"bound": "tensor", "achieved": round(tflops, 3), "peak": round(peak, 1),
                "unit": "TFLOP/s", "frac": round(tflops / peak, 4), "traffic": None,
                "kernel": fam, "peak_source": src + "; achieved counts the 3 TF32 products "
                "per complex product"}
    if fam == "invert" and prec != 0:
        # FP32 blocks are inverted by the tensor-core Gauss-Jordan kernel: its rank-16
        # updates run as 3xTF32 tcgen05 products (3x the algorithmic complex flops, as for the
        # GEMMs); the 16-column panels in between are factored on the FP32 pipe
        tflops = 3.0 * stats["flops"] / (ms * 1e-3) / 1e12
        if live and live.get("tf32_tcgen05_tflops"):
            peak = live["tf32_tcgen05_tflops"]
            src = "measured in this run: tcgen05.mma kind::tf32 128x256 loop on every SM"
        else:
            peak = peaks.get("bf16_tflops_sustained", 1700.0) * TF32_OVER_BF16
            src = f"{peak_kind} sustained bf16 x 1.1/2.25 (TF32)"
        traffic = None
        if ny == 160 and GJ_TC_DRAM_BYTES_PER_BLOCK_NY160:
            blocks = stats["flops"] / (8.0 * ny ** 3)      # 8 ny^3 flops per block inverse
            steps = max(1, stats.get("steps", 1))
            traffic = round(GJ_TC_DRAM_BYTES_PER_BLOCK_NY160 * blocks / steps)
        return {"bound": "tensor", "achieved": round(tflops, 3), "peak": round(peak, 1),
                "unit": "TFLOP/s", "frac": round(tflops / peak, 4), "traffic": traffic,
                "kernel": fam, "peak_source": src + "; achieved counts 3 TF32 products per "
                "complex product (8 n^3 algorithmic flops per block)"}
    if fam in ("gemm", "invert", "level0", "qform"):
        tflops = stats["flops"] / (ms * 1e-3) / 1e12
        if prec == 0 or fam == "qform":
            if live and live.get("fp64_fma_tflops"):
                peak, src = live["fp64_fma_tflops"], "measured in this run: FP64 DFMA loop"
            else:
                peak, src = FP64_NOMINAL_TFLOPS, "FP64 nominal 1.25 TFLOP/s (no measured FP64 peak)"
        elif live and live.get("fp32_fma_tflops"):
            peak, src = live["fp32_fma_tflops"], "measured in this run: FP32 FFMA loop"
        else:
            peak = SM_COUNT * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            src = "FP32 FMA: 152 SMs x 128 lanes x 2 flop x max SM clock"
        traffic = None
        return {"bound": "alu", "achieved": round(tflops, 4 if fam == "qform" else 3),
                "peak": round(peak, 3), "unit": "TFLOP/s", "frac": round(tflops / peak, 4),
                "traffic": traffic, "kernel": fam, "peak_source": src}
    gbs = stats["bytes"] / (ms * 1e-3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    return {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
            "frac": round(gbs / peak, 4), "traffic": None, "kernel": fam,
            "peak_source": f"{peak_kind} HBM copy bandwidth"}


def _cpu_baseline(seed: int, timeout_s: float = 240.0):
    """The oracle as it stands, one cold C2 evaluation of design `seed`, single-threaded, in
    a child process; also returns the oracle's F of that design."""
    code = (
        "import sys,time,json; sys.path.insert(0, %r)\n"
        "import workloads as W\n"
        "from oracle.reciprocal import timed_reciprocal\n"
        "wl = W.c2_collimator(); ws = W.widths(500, %d)\n"
        "F, t = timed_reciprocal(wl, ws)\n"
        "print(json.dumps({'F': F, 'seconds': t}))\n" % (ROOT, seed))
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
              "NUMEXPR_NUM_THREADS", "VECLIB_MAXIMUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                           timeout=timeout_s, env=env)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:  # noqa: BLE001
        return {"value": None, "unit": "evals/s", "cores": 1, "kind": "oracle",
                "sample": f"failed: {type(e).__name__}"}, None
    return {"value": round(1.0 / d["seconds"], 5), "unit": "evals/s", "cores": 1,
            "kind": "oracle", "seconds_per_eval": round(d["seconds"], 3),
            "sample": "one cold evaluation of the full 200-lambda workload (raster, assembly, "
                      "SuperLU factor, double-double refined solve, direct quadratic form), "
                      "single thread, on the design of the first timed GPU evaluation"}, d["F"]


def _bf_worker(args):
    """One host process of the oracle brute-force timing: factor design `seed` of the 200-
    wavelength workload, then the forward solves of its share of the 1000-angle rule."""
    seed, worker, workers, per = args
    import workloads as W
    from oracle.light import quadrature_rule
    from oracle.reciprocal import Evaluation
    wl = W.c2_collimator()
    t0 = time.perf_counter()
    ev = Evaluation(wl, W.widths(wl.grid.n_cells, seed))
    t1 = time.perf_counter()
    theta, _ = quadrature_rule(wl.light, wl.n_angles)
    ev.fom_per_angle(theta[worker::workers][:per])
    return t1 - t0, time.perf_counter() - t1, per


def _cpu_bruteforce(seed: int, per_worker: int = 4, max_workers: int = 8):
    """The oracle's brute-force average (Eq. 6, Sec. 5.2) timed on the host cores: one
    spawned process per core (up to max_workers), each factoring the design once and solving
    per_worker angles of the 1000-angle rule; reports the measured rates and the time 1000
    angles would take on those cores."""
    import multiprocessing as mp
    workers = max(1, min(max_workers, os.cpu_count() or 1))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                            "MKL_NUM_THREADS", "CUDA_VISIBLE_DEVICES")}
    for k in saved:
        os.environ[k] = "" if k == "CUDA_VISIBLE_DEVICES" else "1"
    try:
        ctx = mp.get_context("spawn")
        t0 = time.perf_counter()
        with ctx.Pool(workers) as pool:
            res = pool.map(_bf_worker, [(seed, w, workers, per_worker) for w in range(workers)])
        wall = time.perf_counter() - t0
    except Exception as e:  # noqa: BLE001
        return {"kind": "oracle", "sample": f"failed: {type(e).__name__}: {e}"}
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    fac = statistics.mean(r[0] for r in res)
    per_angle = statistics.mean(r[1] / r[2] for r in res)
    n = sum(r[2] for r in res)
    return {"kind": "oracle", "cores": workers, "angles_sampled": n, "wall_s": round(wall, 2),
            "factor_s": round(fac, 2), "s_per_angle_per_core": round(per_angle, 3),
            "angles_1000_s_extrapolated": round(fac + 1000 / workers * per_angle, 1),
            "sample": f"{workers} processes x {per_worker} angles of the 1000-angle rule on the "
                      "200-wavelength workload, each process factoring the design once "
                      "(SuperLU, single thread) and refining every solve (double-double)"}


def _golden(name: str, seed: int):
    """The oracle's stored values for a full-size design (written by tests/golden/
    make_golden.py, which runs only the oracle), or None."""
    p = os.path.join(ROOT, "tests", "golden", f"{name}_seed{seed}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f)


def _config(nx, ny, unknowns, prec_name, S, ws_):
    return {"workload": WORKLOAD, "nx": nx, "ny": ny, "unknowns": unknowns, "cells": 500,
            "light": "annulus 10-30 deg", "objective": "planewave mode, 0 deg",
            "precision": prec_name, "parallelism": f"replicas x{ws_}",
            "concurrent_evaluations": S}


def run_reference(args):
    """The FP64 CPU oracle on the same workload and metric (time-boxed)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    import workloads as W
    from oracle.reciprocal import timed_reciprocal
    wl = W.WORKLOADS[WORKLOAD]()
    budget = float(os.environ.get("RCI_REFERENCE_BUDGET_S", "150"))
    t_warm = None
    for w in range(min(args.warmup, 1)):
        _, t_warm = timed_reciprocal(wl, W.widths(wl.grid.n_cells, 900000 + w))
    per = t_warm or 15.0
    k_run = max(1, min(args.steps, int(budget // per)))
    times = []
    for k in range(k_run):
        _, t = timed_reciprocal(wl, W.widths(wl.grid.n_cells, 1000 + k))
        times.append(t)
    total = sum(times)
    value = k_run / total
    ms = [t * 1e3 for t in times]
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "evals/s",
        "n_gpus": 1, "steps": args.steps, "steps_run": k_run, "warmup": args.warmup,
        "ms_per_step": round(total / k_run * 1e3, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "p50_ms": round(statistics.median(ms), 2), "p99_ms": round(max(ms), 2),
        "config": dict(_config(4040, 160, 646400, "fp64", 1, 1),
                       l2="no flush: the oracle's LU factors exceed the host caches"),
        "cpu_baseline": {"value": round(value, 5), "unit": "evals/s", "cores": 1,
                         "kind": "oracle",
                         "sample": f"{k_run} of {args.steps} cold evaluations of the full workload "
                                   f"(time-boxed to {budget:.0f} s), single thread"},
        "e2e": {"value": round(value, 5), "unit": "evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import workloads as W
    import paper_2207_10701_gb300 as P
    from paper_2207_10701_gb300 import build as B

    ws_, rank, local = _dist()
    B.build()
    torch.cuda.set_device(local)
    if ws_ > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    peaks, peak_kind = _peaks()
    # arithmetic peaks of this GPU, measured now (the rooflines divide by them)
    live = P.measure_peaks(local) if rank == 0 else None
    wl = W.WORKLOADS[WORKLOAD]()
    prec = P.FP64 if args.prec == "fp64" else P.FP32_REFINE
    nc = wl.grid.n_cells
    K, Wm, S = args.steps, args.warmup, max(1, args.streams)
    seeds = _replica_seeds(rank, K + Wm)
    widths_dev = torch.tensor(np.stack([W.widths(nc, s) for s in seeds]), dtype=torch.float64,
                              device=f"cuda:{local}")
    # S independent evaluators, one stream and one host thread each (evaluations of
    # different designs overlap on the device; each evaluation stays in stream order)
    streams = [torch.cuda.Stream(device=local) for _ in range(S)]
    grids = [P.Grid(wl.grid, prec=prec, device=local, stream=st) for st in streams]
    g = grids[0]

    def run_pass(idx, host_widths=None):
        """Evaluate designs idx[k] (round-robin over the evaluators); returns the device
        time from a common start to the last stream's end, per-evaluation device times,
        the F values and info records in idx order."""
        start = torch.cuda.Event(enable_timing=True)
        start.record(torch.cuda.current_stream())
        for st in streams:
            st.wait_event(start)
        ends = [torch.cuda.Event(enable_timing=True) for _ in streams]
        out = [None] * len(idx)
        per = [0.0] * len(idx)
        errs = []

        def worker(w):
            try:
                gw, st = grids[w], streams[w]
                for k in range(w, len(idx), S):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                    gw.set_design(host_widths[k] if host_widths is not None else widths_dev[idx[k]])
                    gw.factor()
                    out[k] = gw.avg_intensity(wl.objective, wl.light)
                    e1.record(st)
                    e1.synchronize()
                    per[k] = e0.elapsed_time(e1)
                ends[w].record(streams[w])
            except Exception as ex:  # noqa: BLE001
                errs.append(ex)

        ths = [threading.Thread(target=worker, args=(w,)) for w in range(S)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        if errs:
            raise errs[0]
        torch.cuda.synchronize()
        total = max(start.elapsed_time(e) for e in ends)
        return total, per, [o[0] for o in out], [o[1] for o in out]

    run_pass(list(range(Wm)))  # warm-up (every evaluator builds its workspaces)
    torch.cuda.synchronize()
    _barrier(ws_)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = P.kernel_launches()
    torch.cuda.synchronize()
    _barrier(ws_)
    total_ms, per, Fs, infos = run_pass(list(range(Wm, Wm + K)))
    _barrier(ws_)
    launches = P.kernel_launches() - l0
    clk = clocks.stop()
    total_ms = _max_over_ranks(total_ms, ws_)
    value = _replica_value(ws_, K, total_ms)

    # ---- one evaluation with nothing else in flight (first evaluator): its latency, and
    # the per-kernel-family device times (CUDA events around each family inside the
    # library) that the roofline record uses, free of interference from other streams
    K1 = min(K, 20)
    lat1 = []
    g.profile(True)
    for k in range(K1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(streams[0])
        g.set_design(widths_dev[Wm + k])
        g.factor()
        g.avg_intensity(wl.objective, wl.light)
        e1.record(streams[0])
        e1.synchronize()
        lat1.append(e0.elapsed_time(e1))
    prof = g.profile_read()
    g.profile(False)
    lat1.sort()

    # ---- end to end through the public API with host buffers (H2D widths, D2H result)
    widths_host = [np.ascontiguousarray(W.widths(nc, 500_000 + rank * 1000 + k))
                   for k in range(K)]
    torch.cuda.synchronize()
    _barrier(ws_)
    t0 = time.perf_counter()
    _, _, _, e2e_infos = run_pass(list(range(K)), host_widths=widths_host)
    e2e_s = _max_over_ranks(time.perf_counter() - t0, ws_)
    e2e_value = ws_ * K / e2e_s
    e2e_iters = sum(i.refine_iters for i in e2e_infos)
    d2h = 8 + 4 + 8 * (e2e_iters / K + 1 + (1 if prec == P.FP64 else 0))

    line = None
    if rank == 0:
        fams = {f: v for f, v in prof.items() if v["ms"] > 0}
        dom = max(fams, key=lambda f: fams[f]["ms"])
        roof = _roofline(dom, dict(fams[dom], steps=K1), prec, peaks, peak_kind, ny=wl.grid.ny,
                         live=live)
        kernels = {}
        for f, v in fams.items():
            r = _roofline(f, dict(v, steps=K1), prec, peaks, peak_kind, ny=wl.grid.ny, live=live)
            kernels[f] = {"ms_per_step": round(v["ms"] / K1, 4),
                          "share": round(v["ms"] / sum(x["ms"] for x in fams.values()), 4),
                          "launches_per_step": v["launches"] / K1,
                          "bound": r["bound"] if r else None,
                          "achieved": r["achieved"] if r else None,
                          "unit": r["unit"] if r else None, "frac": r["frac"] if r else None}
        ps = sorted(per)
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "evals/s", "n_gpus": ws_,
            "steps": K, "warmup": Wm, "ms_per_step": round(total_ms / K, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64refine" if prec == P.FP32_REFINE else "f64",
            "data": "synthetic",
            "p50_ms": round(ps[len(ps) // 2], 4),
            "p99_ms": round(ps[min(len(ps) - 1, int(math.ceil(0.99 * len(ps))) - 1)], 4),
            "latency_alone": {"p50_ms": round(lat1[len(lat1) // 2], 4),
                              "p99_ms": round(lat1[-1], 4), "evals": len(lat1)},
            "config": dict(_config(g.nx, g.ny, g.N, args.prec, S, ws_),
                           l2="no flush: factor store %.2f GB > 129 MB L2"
                              % (g.device_bytes() / 1e9),
                           refine_iters_mean=round(sum(i.refine_iters for i in infos) / K, 2),
                           rel_residual_max=max(i.rel_residual for i in infos),
                           fp64_fallbacks=sum(1 for i in infos if i.fallback),
                           simt_refactors=sum(1 for i in infos if i.simt_refactor)),
            "measured_peaks": {k: (round(v, 3) if isinstance(v, float) else v)
                               for k, v in (live or {}).items()},
            "gpu_launches": int(launches),
            "roofline": roof,
            "kernels": kernels,
            "clocks": clk,
            "e2e": {"value": round(e2e_value, 3), "unit": "evals/s",
                    "h2d_bytes_per_step": 8 * nc, "d2h_bytes_per_step": int(round(d2h))},
            "F_first": Fs[0],
            "F_last": Fs[-1],
        }
    for gw in grids:
        gw.close()
    stream = streams[0]

    # ---- FP64 form and brute-force comparison (rank 0, outside the timed region)
    if rank == 0 and not args.quick:
        extra = {}
        other = P.FP64 if prec == P.FP32_REFINE else P.FP32_REFINE
        with P.Grid(wl.grid, prec=other, device=local, stream=stream) as g2:
            t = []
            for k in range(args.other_steps + 1):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g2.set_design(widths_dev[Wm + k % K])
                g2.factor()
                F2, _ = g2.avg_intensity(wl.objective, wl.light)
                e1.record(stream)
                torch.cuda.synchronize()
                if k:
                    t.append(e0.elapsed_time(e1))
            t.sort()
            extra["fp64" if other == P.FP64 else "fp32_refine"] = {
                "evals_per_s": round(1e3 / (sum(t) / len(t)), 3), "p50_ms": round(t[len(t) // 2], 3),
                "p99_ms": round(t[-1], 3), "steps": len(t)}
        with P.Grid(wl.grid, prec=prec, device=local, stream=stream) as g3:
            g3.set_design(widths_dev[Wm])
            g3.factor()
            Fr, _ = g3.avg_intensity(wl.objective, wl.light)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            Fb, _, binfo = g3.avg_bruteforce(wl.objective, wl.light, wl.n_angles)
            e1.record(stream)
            torch.cuda.synchronize()
            tb = e0.elapsed_time(e1)
            e0.record(stream)
            Fr2, rinfo = g3.avg_intensity(wl.objective, wl.light)
            e1.record(stream)
            torch.cuda.synchronize()
            tr = e0.elapsed_time(e1)
            extra["bruteforce"] = {
                "angles": wl.n_angles, "ms": round(tb, 2),
                "reciprocal_warm_ms": round(tr, 3),
                "time_ratio_brute_over_reciprocal": round(tb / tr, 1),
                "F_reciprocal": Fr, "F_bruteforce": Fb,
                "rel_diff": abs(Fb - Fr) / abs(Fr)}
        # cold evaluations with the adjoint width gradient on the gradient workload
        # (C2's grid, virtual focus 20 wavelengths up, cone of +-15 degrees)
        wg = W.c4_gradient()
        with P.Grid(wg.grid, prec=prec, device=local, stream=stream) as g4:
            t = []
            for k in range(args.other_steps + 1):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g4.set_design(widths_dev[Wm + k % K])
                g4.factor()
                Fg, grad, ginfo = g4.avg_intensity_grad(wg.objective, wg.light)
                e1.record(stream)
                torch.cuda.synchronize()
                if k:
                    t.append(e0.elapsed_time(e1))
            t.sort()
            extra["gradient"] = {
                "workload": wg.name, "evals_per_s": round(1e3 / (sum(t) / len(t)), 3),
                "p50_ms": round(t[len(t) // 2], 3), "p99_ms": round(t[-1], 3), "steps": len(t),
                "grad_norm_inf": float(np.max(np.abs(grad)))}
            # 100 projected-gradient iterations from seed-0 widths, clamped to [0.08, 0.36]
            from paper_2207_10701_gb300.design import optimize
            t0 = time.perf_counter()
            res = optimize(g4, wg.objective, wg.light, W.widths(wg.grid.n_cells, 0), iters=100,
                           step=0.01)
            extra["design_loop"] = {
                "workload": wg.name, "iterations": len(res.steps), "accepted": len(res.history) - 1,
                "F_start": res.history[0], "F_end": res.history[-1],
                "gain": round(res.history[-1] / res.history[0], 4),
                "seconds": round(time.perf_counter() - t0, 2),
                "evaluations": res.evaluations, "refine_iters_max": res.refine_iters_max,
                "simt_refactors": res.simt_refactors, "fp64_fallbacks": res.fp64_fallbacks}
        # the precision form at 1000 wavelengths (2500 cells, nx 20040, ny 224, 4.5M unknowns,
        # virtual focus 50 wavelengths up, cone of +-20 degrees): cold FP32 + refinement
        # evaluations against the FP64 form of the same design, one grid at a time
        w3 = W.c3_precision()
        ws3 = W.widths(w3.grid.n_cells, 0)
        c3 = {"workload": w3.name}
        for pr, name, reps in ((P.FP32_REFINE, "fp32_refine", 2), (P.FP64, "fp64", 1)):
            with P.Grid(w3.grid, prec=pr, device=local, stream=stream) as g5:
                c3["unknowns"] = g5.N
                t = []
                for k in range(reps + (1 if pr == P.FP32_REFINE else 0)):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    g5.set_design(ws3)
                    g5.factor()
                    F3, info3 = g5.avg_intensity(w3.objective, w3.light)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    if k or pr == P.FP64:
                        t.append(e0.elapsed_time(e1))
                c3[name] = {"ms_per_eval": round(sum(t) / len(t), 2), "F": F3,
                            "refine_iters": info3.refine_iters,
                            "rel_residual": info3.rel_residual, "fp64_fallback": info3.fallback,
                            "device_gb": round(g5.device_bytes() / 1e9, 2)}
        c3["rel_diff_fp32_refine_vs_fp64"] = (abs(c3["fp32_refine"]["F"] - c3["fp64"]["F"])
                                              / abs(c3["fp64"]["F"]))
        gold = _golden(w3.name, 0)
        if gold is not None:
            c3["F_oracle"] = gold["F"]
            for name in ("fp32_refine", "fp64"):
                c3[name]["rel_err_vs_oracle"] = abs(c3[name]["F"] - gold["F"]) / abs(gold["F"])
        extra["c3_precision"] = c3
        line.update(extra)
    if rank == 0 and not args.quick and not args.no_serve_leg:
        line["serving"] = _serving_leg(args, local)
    if rank == 0 and not args.no_cpu_baseline and ws_ == 1:
        # the oracle on the design of the first timed evaluation: its time is the CPU
        # baseline, its F the per-result error of that evaluation
        cb, F_or = _cpu_baseline(Wm)
        if not args.quick:
            cb["bruteforce"] = _cpu_bruteforce(Wm)
        line["cpu_baseline"] = cb
        if F_or is not None:
            line["rel_err_vs_oracle"] = {"F_gpu": Fs[0], "F_oracle": F_or,
                                         "rel_err": abs(Fs[0] - F_or) / abs(F_or),
                                         "tolerance": 1e-8 if prec == P.FP32_REFINE else 1e-9,
                                         "design_seed": Wm}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws_ > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _serve_stream(P, W, local, n_requests, slots, arena_gb, cache_gb, repeat, rate=0.0):
    """Requests with Poisson arrivals (metasurfaces of 50..1250 cells, concentrator /
    collimator, cone / annulus, 30 % with the gradient; `repeat` of them re-evaluating one
    of the last 32 designs under new light) admitted continuously by the library's server.
    The arrival rate defaults to 70 % of the capacity measured on the same requests in a
    closed loop (all submitted at once) on a server of its own, so that the capacity
    reflects this stream's mix -- its large grids and the rare designs that need the FP64
    factorisation -- and the timed run starts with an empty factorisation cache."""
    import numpy as np

    arena = int(arena_gb * (1 << 30))
    cache = int(cache_gb * (1 << 30))

    def run(srv, reqs, paced):
        t_start = time.perf_counter()
        tickets = [None] * len(reqs)

        def submitter():
            for k, r in enumerate(reqs):
                if paced:
                    dt = r.arrival_s - (time.perf_counter() - t_start)
                    if dt > 0:
                        time.sleep(dt)
                tickets[k] = srv.submit(r.grid, r.widths, r.objective, r.light,
                                        want_grad=r.want_grad, design_key=r.design_key)
        th = threading.Thread(target=submitter)
        th.start()
        out = []
        for k in range(len(reqs)):
            while tickets[k] is None:
                time.sleep(0.0005)
            out.append(srv.wait(tickets[k], timeout=3600))
        th.join()
        return out

    def server():
        return P.Server(device=local, slots=slots, arena_bytes=arena, cache_bytes=cache,
                        lookahead=8)

    with server() as srv:
        # warm-up (kernels loaded, arena touched), then the closed-loop capacity
        run(srv, W.serving_requests(16, 0.0, seed=999), paced=False)
        closed = run(srv, W.serving_requests(n_requests, 1.0, seed=1, repeat_fraction=repeat),
                     paced=False)
    span = (max(r["t_end_us"] for r in closed) - min(r["t_submit_us"] for r in closed)) * 1e-6
    capacity = len(closed) / span
    rate = rate if rate > 0 else 0.7 * capacity
    reqs = W.serving_requests(n_requests, rate, seed=1, repeat_fraction=repeat)
    with server() as srv:
        run(srv, W.serving_requests(16, 0.0, seed=999), paced=False)
        st0 = srv.stats()
        clocks = ClockSampler(local)
        clocks.start()
        res = run(srv, reqs, paced=True)
        clk = clocks.stop()
        st = srv.stats()
    lat = np.array([(r["t_end_us"] - r["t_submit_us"]) * 1e-3 for r in res])
    wait = np.array([(r["t_start_us"] - r["t_submit_us"]) * 1e-3 for r in res])
    ok = [r["status"] == 0 for r in res]             # converged to the tolerance
    unconverged = sum(1 for r in res if r["status"] == 6)   # RCI_ENOCONV: value not counted
    status_counts = {}
    for r in res:
        status_counts[str(r["status"])] = status_counts.get(str(r["status"]), 0) + 1
    span = (max(r["t_end_us"] for r in res) - min(r["t_submit_us"] for r in res)) * 1e-6
    grad = np.array([q.want_grad for q in reqs])
    fb = np.array([bool(r.get("fp64_fallback", 0)) for r in res])
    sr = np.array([bool(r.get("simt_refactor", 0)) for r in res])
    delta = ("submitted", "completed", "failed", "admission_waits", "bypasses", "cache_hits",
             "cache_evictions")
    return {
        "value": round(sum(ok) / span, 3), "unit": "evals/s",
        "p50_ms": round(float(np.percentile(lat, 50)), 3),
        "p99_ms": round(float(np.percentile(lat, 99)), 3),
        "p50_queue_ms": round(float(np.percentile(wait, 50)), 3),
        "p99_queue_ms": round(float(np.percentile(wait, 99)), 3),
        "p50_ms_gradient": round(float(np.percentile(lat[grad], 50)), 3) if grad.any() else None,
        "fp64_fallbacks": int(fb.sum()),
        "simt_refactors": int(sr.sum()),
        "p99_ms_fp32_only": round(float(np.percentile(lat[~fb], 99)), 3) if (~fb).any() else None,
        "requests": len(reqs), "failed": len(reqs) - sum(ok), "unconverged": unconverged,
        "status_counts": status_counts, "repeated_designs": round(repeat, 3),
        "arrival_rate_per_s": round(rate, 3), "capacity_evals_per_s": round(capacity, 3),
        "config": {"workload": "serving stream: 50-1250 cells log-uniform, ny 160, "
                               "concentrator/collimator, cone/annulus, 30% gradient",
                   "slots": slots, "arena_gb": arena_gb, "cache_gb": cache_gb, "lookahead": 8,
                   "arrival_rate": "70% of the capacity of a closed-loop run of the same requests"},
        "server": {k: st[k] - st0.get(k, 0) if k in delta else st[k] for k in st},
        "clocks": clk,
    }


def _serving_leg(args, local):
    """The serving form inside the default line: a compact stream (512 requests by default)
    with repeated designs, a factorisation cache and an arena small enough that admission
    has to wait for memory."""
    import workloads as W
    import paper_2207_10701_gb300 as P
    return _serve_stream(P, W, local, args.serve_leg_requests, 6, 24.0, 6.0, 0.25)


def run_serve(args):
    """Serving form as its own line (--serve): the full 4096-request stream."""
    import torch

    import workloads as W
    import paper_2207_10701_gb300 as P
    from paper_2207_10701_gb300 import build as B

    ws_, rank, local = _dist()
    if rank != 0:
        return 0
    B.build()
    torch.cuda.set_device(local)
    d = _serve_stream(P, W, local, args.serve_requests, args.serve_slots,
                      args.serve_arena_gb, args.serve_cache_gb, args.serve_repeat,
                      rate=args.serve_rate)
    line = {"metric": "serving: reciprocal evaluations/s under Poisson arrivals, p50/p99 latency",
            "n_gpus": 1, "higher_is_better": True, "impl": "ours", "dtype": "f32+f64refine",
            "data": "synthetic"}
    line.update(d)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--other-steps", type=int, default=5)
    ap.add_argument("--streams", type=int, default=4,
                    help="independent evaluations in flight (one stream + host thread each)")
    ap.add_argument("--quick", action="store_true", help="skip the FP64 / brute-force extras")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve", action="store_true",
                    help="serving form instead of the evaluation benchmark")
    ap.add_argument("--serve-requests", type=int, default=4096)
    ap.add_argument("--serve-rate", type=float, default=0.0, help="arrivals/s (0: 70%% of capacity)")
    ap.add_argument("--serve-slots", type=int, default=6)
    ap.add_argument("--serve-arena-gb", type=float, default=96.0)
    ap.add_argument("--serve-cache-gb", type=float, default=0.0)
    ap.add_argument("--serve-repeat", type=float, default=0.0,
                    help="fraction of requests re-evaluating a recent design")
    ap.add_argument("--serve-leg-requests", type=int, default=512,
                    help="requests of the serving leg in the default line")
    ap.add_argument("--no-serve-leg", action="store_true")
    args = ap.parse_args()
    if args.serve:
        return run_serve(args)
    if args.impl == "ours":
        args.warmup = max(3, args.warmup)   # never time fewer than 3 warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

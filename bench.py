"""Benchmark of the belief-tensor localizer (Alg. 1 + the Eq. 9 normaliser, Section III-B's
sampled scan update) on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload serve256] [--impl ours]

Default workload (serve256): 256 robot sessions on 10 office plans (256^2 to 2048^2 cells,
K = 36 .. 72 bins) served by the library's serving loop: odometry at 100 Hz per session with
Poisson jitter, a scan at 10 Hz on half of them, admission against a 120 GB budget.  One step
is 100 ms of every session's messages; W steps are submitted and drained untimed, then K steps
are timed.  Four runs on the same message streams:
  * served BF16 (continuous batching, one persistent launch per tick), saturated: every timed
    message submitted at once, so the server's span is its capacity -> `value`;
  * the plain FP32 per-session path (one loc_step per message), saturated -> plain capacity;
  * both again at real-time arrival -> p50 / p99 step latency.
The line also nests the office512 FP32 single-session step (device-timed with CUDA events, L2
flushed before every step) and the office2048 BF16 workload with a sampled scan update every
10th step.  Other workloads (--workload office512, office512_aniso, office512_dense,
office2048, batch64, rooms64) print their own line.  N > 1 runs one independent replica per
rank (weak scaling, no data-path collective); rank 0 prints one JSON line.

--impl reference times the FP64 CPU oracle on the host cores instead (each step a bounded
sample of the same workload: a band of map rows, all bins), printing the same metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the serving loop runs scan updates on up to 32 streams at once; CUDA maps streams onto this
# many hardware work queues (its default is 8), fixed when the process creates its context
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from synth import workloads  # noqa: E402

METRIC = "belief cell-updates/s and p99 step latency, served BF16 vs plain FP32, 1 GB300"
UNIT = "cell-updates/s"
ELEM = {"f32": 4, "bf16": 2, "f16": 2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 60 for serve256, 2000 otherwise)")
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default="serve256")
    ap.add_argument("--storage", default=None, help="override the workload's storage type")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", type=int, default=0, help="tiled-kernel configuration (0: auto)")
    ap.add_argument("--kernel", type=int, default=0, help="0 auto, 1 generic, 2 tiled")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ref-budget-s", type=float, default=150.0,
                    help="CPU seconds the reference arm's timed oracle steps may take together")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed

def dist_init(n):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            if self.uuid and self.uuid not in f[0] and f[0] not in self.uuid:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- CPU oracle

def oracle_band_rate(wl, occ, odom, budget_s: float, steps: int | None = None):
    """Time the FP64 oracle's whole step (Filter.step) on a band of map rows (all bins).
    Returns (cell-updates/s, seconds per step, rows, steps run)."""
    from oracle import aniso as A
    from oracle import filter as F
    H, W, K = wl["H"], wl["W"], wl["K"]

    def make(band):
        if wl.get("sigma_cross_cells", 0.0) > 0.0:
            return A.Filter(band, K, wl["cell"], wl["sigma_xy_cells"], wl["sigma_cross_cells"],
                            wl["sigma_theta_bins"])
        return F.Filter(band, K, wl["cell"], wl["sigma_xy_cells"], wl["sigma_theta_bins"])

    # cost model from a 16-row probe, then size the band to fit the budget
    probe_rows = min(H, 16)
    j0 = (H - probe_rows) // 2
    f = make(occ[j0:j0 + probe_rows])
    t = time.perf_counter()
    f.step(*odom[0])
    per_row = (time.perf_counter() - t) / probe_rows
    n_steps = steps if steps is not None else 2
    rows = int(max(4, min(H, budget_s / max(n_steps, 1) / max(per_row, 1e-9))))
    j0 = (H - rows) // 2
    f = make(occ[j0:j0 + rows])
    times = []
    for s in range(n_steps):
        t = time.perf_counter()
        f.step(*odom[s % len(odom)])
        times.append(time.perf_counter() - t)
    per_step = statistics.mean(times)
    return rows * W * K / per_step, per_step, rows, n_steps, times


# ----------------------------------------------------------------------------- ncu traffic

def profiled_traffic(wl, args):
    """DRAM bytes per launch of the propagation kernel from the committed ncu summary, only
    while the kernel source is the one that was profiled (else None)."""
    import hashlib
    import re
    if wl["name"] != "office512" or wl["storage"] != "f32" or args.tile not in (0, 16) or args.kernel not in (0, 2):
        return None
    try:
        text = open(os.path.join(ROOT, "profiles", "step_ws_office512.md")).read()
        csrc = os.path.join(ROOT, "paper_1910_00572_gb300", "csrc")
        src = b"".join(open(os.path.join(csrc, f), "rb").read() for f in ("tiled_common.cuh", "step_tiled.cu"))
    except OSError:
        return None
    sha = re.search(r"source_sha256:\s*([0-9a-f]+)", text)
    val = re.search(r"dram_bytes_per_launch:\s*([0-9]+)", text)
    if not sha or not val or sha.group(1) != hashlib.sha256(src).hexdigest():
        return None
    return int(val.group(1))


def served_traffic(alg_bytes_per_launch):
    """DRAM bytes per batched launch of the served workload: the ratio of DRAM to algorithmic
    bytes that the committed ncu summary measured on a batched launch (batch64: the same kernel
    source, a smaller workload that ncu can capture in full), times this run's algorithmic bytes
    per launch, only while the batched kernel's source is the one that was profiled (else None).
    The kernel reads each input plane once and writes each output once, so its traffic grows in
    proportion to the cell-updates of the launch."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", "batch_kernel_batch64_bf16.md")).read()
        csrc = os.path.join(ROOT, "paper_1910_00572_gb300", "csrc")
        src = b"".join(open(os.path.join(csrc, f), "rb").read() for f in ("tiled_common.cuh", "batch.cu"))
    except OSError:
        return None
    sha = re.search(r"source_sha256:\s*([0-9a-f]+)", text)
    ratio = re.search(r"dram_per_algorithmic_byte:\s*([0-9.]+)", text)
    if not sha or not ratio or sha.group(1) != hashlib.sha256(src).hexdigest() or not alg_bytes_per_launch:
        return None
    return float(ratio.group(1)) * alg_bytes_per_launch


# ----------------------------------------------------------------------------- arms

def run_reference(args, wl, occ, walk, ws, rank):
    if rank != 0:
        return
    K_, W_ = args.steps, args.warmup
    budget = 150.0
    rate, per_step, rows, n, times = oracle_band_rate(wl, occ, walk.odom, budget, steps=K_ + W_)
    timed = times[W_:] if len(times) > W_ else times
    sec = statistics.mean(timed)
    cells = rows * wl["W"] * wl["K"]
    value = cells / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": K_, "warmup": W_, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(wl, args, extra={"sample": f"oracle step on a {rows}-row band"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"FP64 oracle Filter.step on rows {rows} x {wl['W']} x "
                                   f"{wl['K']} bins of the same map, {len(timed)} timed steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(wl, args, extra=None):
    c = {"workload": wl["name"], "H": wl["H"], "W": wl["W"], "K": wl["K"], "cell_m": wl["cell"],
         "storage": wl["storage"], "sigma_xy_cells": wl["sigma_xy_cells"],
         "sigma_theta_bins": wl["sigma_theta_bins"], "global_batch": 1,
         "sigma_cross_cells": wl.get("sigma_cross_cells", 0.0),
         "parallelism": f"replicas{args.gpus}" if args.gpus > 1 else "single",
         "l2": "flushed (512 MiB device write) before every timed step"}
    if extra:
        c.update(extra)
    return c


def run_ours(args, wl, occ, walk, ws, rank, local):
    line = measure_single(args, wl, occ, walk, ws, rank, local)
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_single(args, wl, occ, walk, ws, rank, local, cpu_budget_s=15.0):
    """One session stepped K times (device-timed, L2 flushed before every step), then the same
    end to end through the C-ABI; the JSON line of the single-session workloads (rank 0; None
    on the other ranks)."""
    import torch

    import paper_1910_00572_gb300 as loc
    from paper_1910_00572_gb300 import build
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    storage = wl["storage"]
    p = loc.loc_params_default(H=wl["H"], W=wl["W"], K=wl["K"], cell_m=wl["cell"],
                               sigma_xy_cells=wl["sigma_xy_cells"],
                               sigma_theta_bins=wl["sigma_theta_bins"], storage=storage,
                               sigma_cross_cells=wl.get("sigma_cross_cells", 0.0),
                               stream=loc.torch_stream(), tile=args.tile, kernel=args.kernel)
    h = loc.loc_create(occ, p)
    odom = walk.odom
    n_cells = wl["H"] * wl["W"] * wl["K"]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    try:
        for s in range(args.warmup):
            loc.loc_step(h, *odom[s % len(odom)])
        torch.cuda.synchronize()
        barrier(ws)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        uuid = None
        try:
            uuid = str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            pass
        with ClockSampler(uuid) as clk:
            torch.cuda.synchronize()
            for s in range(args.steps):
                flush.zero_()
                starts[s].record()
                loc.loc_step(h, *odom[(args.warmup + s) % len(odom)])
                ends[s].record()
            torch.cuda.synchronize()
        loc.loc_sync(h)
        barrier(ws)
        ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        total_s = max_over_ranks(sum(ms) / 1e3, ws)
        per_step_s = total_s / args.steps
        value = n_cells * ws / per_step_s
        p50, p99 = float(np.percentile(ms, 50)), float(np.percentile(ms, 99))

        # end to end through the C-ABI: odometry in, pose estimate (argmax) out, every step
        n_e2e = 0 if args.no_e2e else min(args.steps, 1000)
        e2e_t = 0.0
        for s in range(n_e2e):
            flush.zero_()
            torch.cuda.synchronize()
            t = time.perf_counter()
            loc.loc_step(h, *odom[s % len(odom)])
            loc.loc_argmax(h)
            e2e_t += time.perf_counter() - t
        e2e_t = max_over_ranks(e2e_t, ws)
        e2e_value = n_cells * ws * n_e2e / e2e_t if n_e2e else None
        # the readback of the pose estimate: argmax, mass near it, second hypothesis (device time)
        est_ms = []
        for _ in range(20):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            loc.loc_estimate(h, 0.5, 2)
            e1.record()
            torch.cuda.synchronize()
            est_ms.append(e0.elapsed_time(e1))
        stats = loc.loc_stats(h)
    finally:
        loc.loc_destroy(h)

    if rank != 0:
        return None
    elem = ELEM[storage]
    aniso = wl.get("sigma_cross_cells", 0.0) > 0.0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    if aniso:
        # ALU-bound: the FP32 operations the definition takes per output cell (the theta sum,
        # the rotated x/y stencil over C_k and over the map for G_k, the bilinear pull) against
        # 152 SMs x 128 FP32 lanes x 2 flop x the maximum SM clock of 2070 MHz
        side = 2 * math.ceil(3 * max(wl["sigma_xy_cells"], wl["sigma_cross_cells"])) + 1
        rt = math.ceil(3 * wl["sigma_theta_bins"])
        flops_cell = 2 * ((2 * rt + 1) + 2 * side * side + 4)
        achieved = n_cells * flops_cell / (statistics.mean(ms) / 1e3) / 1e12
        peak = 152 * 128 * 2 * 2.070e9 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "step_aniso (fused propagation with the per-bin rotated stencil + normaliser)",
                "algorithmic_flops_per_launch": n_cells * flops_cell,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}
    else:
        alg_bytes = n_cells * 2 * elem + wl["H"] * wl["W"] * (1 + 4)
        achieved = alg_bytes / (statistics.mean(ms) / 1e3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": profiled_traffic(wl, args),
                "kernel": "step (fused propagation + normaliser)",
                "algorithmic_bytes_per_launch": alg_bytes,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback"}
    cpu = None
    if ws == 1 and not args.no_cpu_baseline and cpu_budget_s > 0:
        rate, per_step, rows, n, _ = oracle_band_rate(wl, occ, odom, budget_s=cpu_budget_s, steps=2)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"FP64 oracle Filter.step on a {rows}-row band ({rows} x {wl['W']} x "
                         f"{wl['K']} cells) of the same map, mean of {n} steps, "
                         f"{per_step:.2f} s/step"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": storage, "data": "synthetic",
        "config": config_of(wl, args, extra={"tile": args.tile, "kernel": args.kernel}),
        "p50_step_ms": p50, "p99_step_ms": p99,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 16 * wl["K"],
                "d2h_bytes_per_step": 12, "steps": n_e2e,
                "path": "loc_step (odometry -> per-bin shift table in the launch parameters) + "
                        "loc_argmax (pose estimate read back), host wall clock"},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "last_Z": stats["last_Z"],
        "estimate_readback": {"ms": float(np.median(est_ms)), "kernels": "argmax + estimate (two passes)",
                              "achieved_gbs": 2 * n_cells * elem / (float(np.median(est_ms)) / 1e3) / 1e9,
                              "note": "device time of loc_estimate(0.5 m, 2 bins) incl. its pinned readback"},
    }
    return line


# ----------------------------------------------------------------------------- many sessions

def session_params(loc, s, storage, **kw):
    return loc.loc_params_default(H=s["H"], W=s["W"], K=s["K"], cell_m=s["cell"], storage=storage, **kw)


def read_peak():
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return peaks["hbm_gbs"], "MEASURED_PEAKS.json hbm_gbs"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def run_batch64(args, wl, ws, rank, local):
    """64 sessions of uneven size: one persistent batched launch per tick (autotuned tiles, CUDA
    graph) against the plain path (one loc_step launch per session), FP32 and BF16."""
    import torch

    import paper_1910_00572_gb300 as loc
    from paper_1910_00572_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    steps = min(args.steps, 300)
    sess = workloads.make_sessions(wl, steps + args.warmup)
    cells = sum(s["H"] * s["W"] * s["K"] for s in sess)
    hw = sum(s["H"] * s["W"] for s in sess)
    odo = np.stack([s["odom"] for s in sess], axis=1)          # [t][session][3]
    res = {}
    clk_summary = None
    storages = ("f32", "bf16") if args.storage is None else (args.storage,)
    for storage in storages:
        hs = [loc.loc_create(s["occ"], session_params(loc, s, storage)) for s in sess]
        try:
            b = loc.loc_batch_create(hs, tile=args.tile if 0 < args.tile <= loc.LOC_BATCH_CONFIGS else 0,
                                     use_graph=True)
            info = loc.loc_batch_info(b)
            try:
                def batch_tick(t):
                    loc.loc_batch_step(b, odo[t, :, 0], odo[t, :, 1], odo[t, :, 2])

                def singles_tick(t):
                    for q, h in enumerate(hs):
                        loc.loc_step(h, *odo[t, q])

                out = {}
                for name, tick in (("batched", batch_tick), ("singles", singles_tick)):
                    for t in range(args.warmup):
                        tick(t)
                    torch.cuda.synchronize()
                    barrier(ws)
                    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
                    with ClockSampler(None) as clk:
                        ev[0].record()
                        for t in range(steps):
                            tick(args.warmup + t)
                            ev[t + 1].record()
                        torch.cuda.synchronize()
                    ms = [ev[t].elapsed_time(ev[t + 1]) for t in range(steps)]
                    total = max_over_ranks(ev[0].elapsed_time(ev[steps]) / 1e3, ws)
                    out[name] = {"ms_per_tick": total / steps * 1e3, "value": cells * ws * steps / total,
                                 "p50_tick_ms": float(np.percentile(ms, 50)),
                                 "p99_tick_ms": float(np.percentile(ms, 99))}
                    if name == "batched":
                        clk_summary = clk.summary()
                loc.loc_batch_sync(b)
                # end to end: odometry from host arrays in, every session's pose estimate out
                n_e2e = 0 if args.no_e2e else min(steps, 50)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for t in range(n_e2e):
                    batch_tick(t)
                    for h in hs:
                        loc.loc_argmax(h)
                e2e_t = max_over_ranks(time.perf_counter() - t0, ws)
                out["e2e"] = cells * ws * n_e2e / e2e_t if n_e2e else None
                out["tile"] = info["tile"]
                out["tune_ms"] = info["tune_ms"]
                out["grid"] = info["grid"]
            finally:
                loc.loc_batch_destroy(b)
        finally:
            for h in hs:
                loc.loc_destroy(h)
        res[storage] = out
    if rank != 0:
        return
    peak, src = read_peak()
    head = "bf16" if "bf16" in res else storages[0]
    bf = res[head]
    elem = ELEM[head]
    alg_bytes = cells * 2 * elem + hw * 5
    achieved = alg_bytes / (bf["batched"]["ms_per_tick"] / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": bf["batched"]["value"], "unit": UNIT, "n_gpus": ws, "steps": steps,
        "warmup": args.warmup, "ms_per_step": bf["batched"]["ms_per_tick"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": head, "data": "synthetic",
        "config": {"workload": "batch64", "sessions": len(sess), "cells_per_tick": cells,
                   "sides": sorted({s["H"] for s in sess}), "K": sorted({s["K"] for s in sess}),
                   "global_batch": len(sess), "parallelism": f"replicas{ws}" if ws > 1 else "single",
                   "l2": "inputs larger than L2 (every tick reads and writes all sessions' tensors)"},
        "p50_step_ms": bf["batched"]["p50_tick_ms"], "p99_step_ms": bf["batched"]["p99_tick_ms"],
        "batched_vs_singles": res,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "batch (persistent propagation over all sessions)",
                     "algorithmic_bytes_per_launch": alg_bytes, "peak_source": src},
        "cpu_baseline": None,
        "e2e": {"value": bf["e2e"], "unit": UNIT, "h2d_bytes_per_step": 24 * len(sess),
                "d2h_bytes_per_step": 12 * len(sess),
                "path": "loc_batch_step (host odometry arrays) + loc_argmax of every session, host wall clock"},
        "gpu_launches": steps,
        "clocks": clk_summary,
    }
    print(json.dumps(line), flush=True)


def serve_schedule(wl, sess, duration, rng):
    """Message times: odometry at odom_hz per session with exponential jitter (Poisson
    arrivals), a scan with every (odom_hz / scan_hz)-th odometry message of even sessions."""
    per = int(round(wl["odom_hz"] / wl["scan_hz"]))
    odo_t, odo_s, odo_i = [], [], []
    scans = []
    for q, s in enumerate(sess):
        n = len(s["odom"])
        t = np.cumsum(rng.exponential(1.0 / wl["odom_hz"], n))
        k = int(np.searchsorted(t, duration))
        odo_t.append(t[:k])
        odo_s.append(np.full(k, q))
        odo_i.append(np.arange(k))
        if q % 2 == 0:
            for i in range(per - 1, k, per):
                scans.append((float(t[i]) + 1e-6, q, i))
    odo_t, odo_s, odo_i = (np.concatenate(x) for x in (odo_t, odo_s, odo_i))
    order = np.argsort(odo_t, kind="stable")
    scans.sort()
    return odo_t[order], odo_s[order], odo_i[order], scans


WINDOW_S = 0.1        # one step of the served workload: 100 ms of every session's messages


def serve_streams(wl, sess, windows, rng):
    """The message streams of the first `windows` steps (odometry at odom_hz per session with
    Poisson jitter, a scan with every (odom_hz / scan_hz)-th odometry message of even
    sessions) and a pool of four simulated scans per scanning session along its walk."""
    from synth import scan as synth_scan
    duration = windows * WINDOW_S
    odo_t, odo_s, odo_i, scans = serve_schedule(wl, sess, duration, rng)
    pool = {}
    for q, s in enumerate(sess):
        if q % 2 == 0:
            idx = np.linspace(0, min(len(s["poses"]) - 1, int(duration * wl["odom_hz"])), 4).astype(int)
            pool[q] = [synth_scan.simulate_scan(s["occ"], s["cell"], s["poses"][i], seed=q * 7 + j,
                                                n_beams=wl["n_beams"], angle_inc=wl["angle_inc"],
                                                r_max=wl["r_max"], noise_sigma=wl["scan_noise"],
                                                dropout=wl["dropout"], march=0.25)
                       for j, i in enumerate(idx)]
    return odo_t, odo_s, odo_i, scans, pool


def serve_run(loc, wl, sess, streams, storage, batching, realtime, warm_windows, timed_windows, e2e=False):
    """One run of the serving loop on the message streams: the first warm_windows steps are
    submitted at once and drained (untimed), then the next timed_windows steps either at their
    arrival times (realtime) or all at once (saturated: the server's capacity).  Returns the
    server's statistics of the timed part; with e2e, also the client's wall clock from the
    first timed submission to every session's pose read back (loc_argmax) after the drain."""
    odo_t, odo_s, odo_i, scans, pool = streams
    odom = [s["odom"] for s in sess]
    per_session = max(1, int((warm_windows + timed_windows) * WINDOW_S * wl["odom_hz"]))
    srv = loc.loc_server_create(loc.loc_server_params_default(
        hbm_budget_bytes=wl["hbm_budget_gb"] * 1e9, storage=storage, batching=batching, tile=0))
    try:
        ids = [loc.loc_server_open(srv, s["occ"], session_params(loc, s, storage,
                                                                  min_shift_cells=wl["min_shift_cells"],
                                                                  n_samples=wl["n_samples"]))
               for s in sess]
        loc.loc_server_drain(srv, 900.0)                      # admissions (and the autotuner) first
        st0 = loc.loc_server_stats(srv)
        ids_a = np.asarray(ids, np.int32)
        u = np.array([odom[q][i][0] for q, i in zip(odo_s, odo_i)])
        v = np.array([odom[q][i][1] for q, i in zip(odo_s, odo_i)])
        w = np.array([odom[q][i][2] for q, i in zip(odo_s, odo_i)])
        t_split = warm_windows * WINDOW_S
        n_warm = int(np.searchsorted(odo_t, t_split, side="left"))
        sc_warm = int(np.searchsorted([x[0] for x in scans], t_split, side="left"))
        admitted = {q for q in range(len(sess)) if loc.loc_server_session(srv, ids[q])[0] == loc.LOC_SESSION_ACTIVE}
        bytes_in = {"odometry": 0, "scans": 0}

        def submit(j0, j1, sc0, sc1, t0):
            """Messages [j0, j1) and scans [sc0, sc1), in arrival order; t0 None: all at once,
            else each when its time (t0 + its offset) has come.  The server stamps a message's
            arrival when it is submitted, so the latencies are the server's own, from receipt
            to the end of the message's device work."""
            j, sc = j0, sc0

            def odometry_upto(k):
                nonlocal j
                if k > j:
                    loc.loc_server_odometry(srv, ids_a[odo_s[j:k]], u[j:k], v[j:k], w[j:k],
                                            None)
                    bytes_in["odometry"] += (k - j) * (4 + 3 * 8)      # id + (u, v, w)
                    j = k
            while j < j1 or sc < sc1:
                now = loc.loc_server_now(srv) - t0 + t_split if t0 is not None else float("inf")
                while sc < sc1 and scans[sc][0] <= now:
                    ts, q, i = scans[sc]
                    odometry_upto(min(j1, int(np.searchsorted(odo_t, ts, side="right"))))
                    z = pool[q][min(3, 4 * i // per_session)]
                    loc.loc_server_scan(srv, ids[q], z, 0.0, wl["angle_inc"], wl["r_max"], wl["beam_stride"],
                                        wl["sigma_r"], -1.0)
                    bytes_in["scans"] += z.size * 4
                    sc += 1
                odometry_upto(min(j1, int(np.searchsorted(odo_t, now, side="right"))) if t0 is not None else j1)
                if t0 is not None and (j < j1 or sc < sc1):
                    time.sleep(0.0005)

        submit(0, n_warm, 0, sc_warm, None)                   # warm-up: untimed
        loc.loc_server_drain(srv, 900.0)
        loc.loc_server_reset_stats(srv)
        bytes_in["odometry"] = bytes_in["scans"] = 0
        import torch
        with ClockSampler(None) as clk:
            if e2e:
                torch.cuda.profiler.start()      # marks the headline run's timed region for a profiler
            c0 = time.perf_counter()
            t0 = loc.loc_server_now(srv) + 0.02 if realtime else None
            submit(n_warm, len(odo_t), sc_warm, len(scans), t0)
            loc.loc_server_drain(srv, 900.0)
            if e2e:
                torch.cuda.profiler.stop()
            poses = 0
            if e2e:
                for q in sorted(admitted):
                    _, h = loc.loc_server_session(srv, ids[q])
                    loc.loc_argmax(h)
                    poses += 1
            wall = time.perf_counter() - c0
        st = loc.loc_server_stats(srv)
    finally:
        loc.loc_server_destroy(srv)
    span = max(st["last_s"] - st["first_s"], 1e-9)
    out = {"storage": storage, "path": "batched" if batching else "plain (one loc_step per message)",
           "arrival": "realtime" if realtime else "saturated (every message at once)",
           "admitted": st0["n_active"], "pending": st0["n_pending"], "bytes_used_gb": st0["bytes_used"] / 1e9,
           "value": st["cell_updates"] / span, "span_s": span, "ms_per_window": span / timed_windows * 1e3,
           "propagations": st["n_propagations"], "scans": st["n_scans"], "messages": st["n_messages"],
           "mean_batch": st["mean_batch"], "step_p50_ms": st["step_p50_ms"], "step_p99_ms": st["step_p99_ms"],
           "step_max_ms": st["step_max_ms"], "scan_p50_ms": st["scan_p50_ms"], "scan_p99_ms": st["scan_p99_ms"],
           "clocks": clk.summary(),
           "breakdown_ms": {"batch_device": st["batch_device_ms"], "n_batches": st["n_batches"],
                            "scan_device": st["scan_device_ms"], "n_scans": st["n_scans_timed"],
                            "plain_device": st["plain_device_ms"], "n_plain": st["n_plain"],
                            "host_gather": st["host_gather_ms"], "host_batch": st["host_batch_ms"],
                            "host_scan": st["host_scan_ms"], "host_plain": st["host_plain_ms"]},
           "device_bytes": {"batch": st["batch_alg_bytes"], "plain": st["plain_alg_bytes"]}}
    if e2e:
        out["e2e"] = {"value": st["cell_updates"] / wall, "wall_s": wall, "poses_read": poses,
                      "h2d_bytes": bytes_in["odometry"] + bytes_in["scans"], "d2h_bytes": 12 * poses}
    return out


def serve_compare(args, wl, ws, rank, local):
    """The served BF16 form against the plain FP32 per-session path on the same message streams,
    each at capacity (saturated) and at real-time arrival."""
    import torch

    import paper_1910_00572_gb300 as loc
    from paper_1910_00572_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    windows = args.warmup + args.steps
    sess = workloads.make_sessions(wl, int(windows * WINDOW_S * wl["odom_hz"] * 1.5) + 50)
    rng = np.random.Generator(np.random.PCG64(wl["seed"] + 991))
    streams = serve_streams(wl, sess, windows, rng)
    res = {}
    res["bf16_capacity"] = serve_run(loc, wl, sess, streams, "bf16", 1, False, args.warmup, args.steps, e2e=True)
    res["f32_plain_capacity"] = serve_run(loc, wl, sess, streams, "f32", 0, False, args.warmup, args.steps)
    res["bf16_realtime"] = serve_run(loc, wl, sess, streams, "bf16", 1, True, args.warmup, args.steps)
    res["f32_plain_realtime"] = serve_run(loc, wl, sess, streams, "f32", 0, True, args.warmup, args.steps)
    return res, sess


def measure_office2048_scans(args, ws, rank, local):
    """The 2048 x 2048 x 72 BF16 workload as specified: odometry steps with a sampled LIDAR update
    (Floyd-Steinberg samples, ray casts, Eq. 9 reweighting) on every 10th step.  Propagations and
    scan updates are timed separately with CUDA events on the session's stream, L2 flushed
    before each; the step kernel's roofline is the propagation's."""
    import torch

    import paper_1910_00572_gb300 as loc
    from synth import scan as synth_scan
    wl = workloads.get("office2048")
    occ = workloads.make_map(wl)
    n = args.warmup + args.steps
    walk = workloads.make_walk(wl, occ, steps=n)
    dev = torch.device("cuda", local)
    p = loc.loc_params_default(H=wl["H"], W=wl["W"], K=wl["K"], cell_m=wl["cell"], storage=wl["storage"],
                               n_samples=wl["n_samples"], stream=loc.torch_stream())
    h = loc.loc_create(occ, p)
    every = wl["scan_every"]
    scans = {t: synth_scan.simulate_scan(occ, wl["cell"], walk.poses[t], seed=wl["seed"] * 7919 + t,
                                         n_beams=wl["n_beams"], angle_inc=wl["angle_inc"], r_max=wl["r_max"],
                                         noise_sigma=wl["scan_noise"], dropout=wl["dropout"], march=0.25)
             for t in range(every, n + 1, every)}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    step_ms, scan_ms = [], []
    try:
        with ClockSampler(None) as clk:
            for t in range(1, n + 1):
                timed = t > args.warmup
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                loc.loc_step(h, *walk.odom[t - 1])
                e1.record()
                if t in scans:
                    flush.zero_()
                    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e2.record()
                    loc.loc_lidar_update(h, scans[t], 0.0, wl["angle_inc"], wl["r_max"], wl["beam_stride"],
                                         wl["sigma_r"])
                    e3.record()
                torch.cuda.synchronize()
                if timed:
                    step_ms.append(e0.elapsed_time(e1))
                    if t in scans:
                        scan_ms.append(e2.elapsed_time(e3))
        loc.loc_sync(h)
        k, j, i, pmax = loc.loc_argmax(h)
    finally:
        loc.loc_destroy(h)
    cells = wl["H"] * wl["W"] * wl["K"]
    alg = cells * 2 * ELEM[wl["storage"]] + wl["H"] * wl["W"] * 5
    peak, src = read_peak()
    mean_step = statistics.mean(step_ms)
    total = sum(step_ms) + sum(scan_ms)
    return {"workload": "office2048", "H": wl["H"], "W": wl["W"], "K": wl["K"], "storage": wl["storage"],
            "scan_every": every, "steps": len(step_ms), "scans": len(scan_ms),
            "value": cells * len(step_ms) / (total / 1e3),
            "unit": "cell-updates/s (propagations over the time of propagations and scan updates)",
            "step_ms": mean_step, "step_p50_ms": float(np.percentile(step_ms, 50)),
            "step_p99_ms": float(np.percentile(step_ms, 99)),
            "scan_ms": statistics.mean(scan_ms) if scan_ms else None,
            "scan_p99_ms": float(np.percentile(scan_ms, 99)) if scan_ms else None,
            "scan_share": sum(scan_ms) / total if total > 0 else None,
            "roofline": {"bound": "hbm", "achieved": alg / (mean_step / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / (mean_step / 1e3) / 1e9 / peak, "traffic": None,
                         "kernel": "step (fused propagation + normaliser), session default tile",
                         "algorithmic_bytes_per_launch": alg, "peak_source": src},
            "argmax": [k, j, i], "clocks": clk.summary(),
            "l2": "flushed (512 MiB device write) before every timed propagation and scan update"}


def run_office2048_scans(args, ws, rank, local):
    """Config 2 as specified on its own line: 2048 x 2048 x 72 BF16 steps with a sampled scan
    update every 10th step (value: cell-updates/s over the time of propagations and scans)."""
    import torch

    from paper_1910_00572_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    r = measure_office2048_scans(args, ws, rank, local)
    if rank != 0:
        return
    n_total = (r["step_ms"] * r["steps"] + (r["scan_ms"] or 0.0) * r["scans"]) / max(r["steps"], 1)
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": n_total, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "office2048_scans", "H": r["H"], "W": r["W"], "K": r["K"], "storage": r["storage"],
                   "scan_every": r["scan_every"], "global_batch": 1,
                   "parallelism": f"replicas{ws}" if ws > 1 else "single", "l2": r["l2"]},
        "p50_step_ms": r["step_p50_ms"], "p99_step_ms": r["step_p99_ms"],
        "scan_ms": r["scan_ms"], "scan_p99_ms": r["scan_p99_ms"], "scan_share": r["scan_share"],
        "roofline": r["roofline"], "cpu_baseline": None,
        "e2e": None, "gpu_launches": None, "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_serve(wl, sess, budget_s=12.0):
    """The oracle on one session of the mix (session 0, its map and K), as it stands: the FP64
    propagation restated in C (oracle.cprop, bit-identical to the numpy definition) on one core
    and on all host cores, each on a band of map rows sized to the budget, plus the numpy
    definition on one core.  Returns the cpu_baseline object (value = all cores)."""
    import platform

    from oracle import cprop
    from oracle import filter as F
    s = sess[0]
    occ, K = s["occ"], s["K"]
    H, W = occ.shape
    cores = cprop.host_cores()
    odo = s["odom"]

    def band_rate(make, per_cell_guess, budget):
        rows = int(max(8, min(H, budget / 2 / max(per_cell_guess * W * K, 1e-12))))
        j0 = (H - rows) // 2
        f = make(occ[j0:j0 + rows])
        ts = []
        for t in range(2):
            t1 = time.perf_counter()
            f.step(*odo[t])
            ts.append(time.perf_counter() - t1)
        return rows * W * K / statistics.mean(ts), rows, statistics.mean(ts)

    # per-cell cost from a small probe, then a band sized to the budget
    def probe(make):
        f = make(occ[(H - 8) // 2:(H - 8) // 2 + 8])
        t1 = time.perf_counter()
        f.step(*odo[0])
        return (time.perf_counter() - t1) / (8 * W * K)

    mk1 = lambda band: cprop.Filter(band, K, s["cell"], threads=1)           # noqa: E731
    mkn = lambda band: cprop.Filter(band, K, s["cell"], threads=cores)       # noqa: E731
    mknp = lambda band: F.Filter(band, K, s["cell"])                        # noqa: E731
    r1, rows1, t1 = band_rate(mk1, probe(mk1), budget_s / 3)
    rn, rowsn, tn = band_rate(mkn, probe(mkn), budget_s / 3)
    rnp, rowsnp, tnp = band_rate(mknp, probe(mknp), budget_s / 3)
    cpu = platform.processor() or platform.machine()
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                cpu = ln.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"value": rn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle step (propagation restated in C, OpenMP over bins, {cores} threads) on a "
                      f"{rowsn}-row band of session 0 ({H} x {W} map, K = {K}), mean of 2 steps, {tn:.2f} s/step",
            "single_core": {"value": r1, "rows": rows1, "s_per_step": t1, "impl": "oracle.cprop, 1 thread"},
            "numpy_single_core": {"value": rnp, "rows": rowsnp, "s_per_step": tnp,
                                  "impl": "oracle.filter (numpy definition), 1 core"},
            "host": {"nproc": os.cpu_count(), "cores_available": cores, "cpu": cpu, "machine": platform.machine()}}


def headline_config(wl, sess, ws):
    return {"workload": "serve256", "sessions": len(sess), "maps": wl["n_maps"],
            "step": f"{WINDOW_S * 1e3:.0f} ms of every session's messages",
            "odom_hz": wl["odom_hz"], "scan_hz": wl["scan_hz"], "hbm_budget_gb": wl["hbm_budget_gb"],
            "min_shift_cells": wl["min_shift_cells"], "n_samples": wl["n_samples"],
            "cells_all_sessions": sum(s["H"] * s["W"] * s["K"] for s in sess),
            "global_batch": len(sess), "parallelism": f"replicas{ws}" if ws > 1 else "single",
            "l2": "inputs larger than L2 (98 GB of resident belief tensors)",
            "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS")}


def run_headline(args, wl, ws, rank, local):
    """The default line: 256 robot sessions on 10 maps, served BF16 against the plain FP32
    per-session path (value = served BF16 capacity), with the office512 FP32 and office2048
    BF16 (with scans) single-session results nested."""
    res, sess = serve_compare(args, wl, ws, rank, local)
    single = None
    wl1 = workloads.get("office512")
    occ1 = workloads.make_map(wl1)
    walk1 = workloads.make_walk(wl1, occ1, seed_offset=rank)
    single = measure_single(args, wl1, occ1, walk1, ws, rank, local, cpu_budget_s=0.0)
    scans2 = measure_office2048_scans(args, ws, rank, local)
    if rank != 0:
        return
    cap, plain = res["bf16_capacity"], res["f32_plain_capacity"]
    rt, prt = res["bf16_realtime"], res["f32_plain_realtime"]
    peak, src = read_peak()
    bd = cap["breakdown_ms"]
    achieved = cap["device_bytes"]["batch"] / (bd["batch_device"] / 1e3) / 1e9 if bd["batch_device"] > 0 else None
    cpu = cpu_baseline_serve(wl, sess) if (ws == 1 and not args.no_cpu_baseline) else None
    e2e = cap["e2e"]
    line = {
        "metric": METRIC, "value": cap["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": cap["ms_per_window"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": headline_config(wl, sess, ws),
        "value_is": "served BF16 capacity: every timed message submitted at once, cell-updates over the "
                    "server's span from the first arrival to the last completion",
        "plain_f32_capacity": plain["value"],
        "capacity_ratio_bf16_over_f32": cap["value"] / plain["value"] if plain["value"] else None,
        "p50_step_ms": rt["step_p50_ms"], "p99_step_ms": rt["step_p99_ms"],
        "latency_is": "served BF16 at real-time arrival (bf16_realtime): odometry arrival to the end of "
                      "its propagation",
        "runs": res,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None,
                     "traffic": served_traffic(cap["device_bytes"]["batch"] / max(bd["n_batches"], 1)),
                     "traffic_is": "DRAM bytes per launch: the DRAM / algorithmic byte ratio of a batched "
                                   "launch captured by ncu (batch64, same kernel source: "
                                   "profiles/batch_kernel_batch64_bf16.md) times this run's algorithmic bytes "
                                   "per launch",
                     "kernel": "batch (persistent propagation of every session the tick propagates)",
                     "algorithmic_bytes_per_launch": cap["device_bytes"]["batch"] / max(bd["n_batches"], 1),
                     "launches": bd["n_batches"], "peak_source": src,
                     "timing": "CUDA events around each batched tick on the batch stream (table copy + kernel)"},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e["value"], "unit": UNIT,
                "h2d_bytes_per_step": e2e["h2d_bytes"] / args.steps, "d2h_bytes_per_step": e2e["d2h_bytes"] / args.steps,
                "path": "loc_server_odometry / loc_server_scan from host arrays (every timed message at once), "
                        "loc_server_drain, then every admitted session's pose read back (loc_argmax); "
                        "host wall clock"},
        # a batched launch per tick; per scan update: restart check, belief map, dithering, row
        # scan, compaction, scoring and the four reweighting kernels
        "gpu_launches": bd["n_batches"] + 10 * bd["n_scans"],
        "clocks": cap["clocks"],
        "office512_f32": single,
        "office2048_bf16_scans": scans2,
    }
    print(json.dumps(line), flush=True)


def run_reference_serve(args, wl, ws, rank):
    """The oracle arm of the default workload: the oracle as it stands (FP64 propagation restated
    in C on all host cores) stepping session 0 of the mix, K timed steps after W warm-up steps,
    each on a band of map rows (a bounded sample)."""
    if rank != 0:
        return
    from oracle import cprop
    sess = workloads.make_sessions(wl, args.warmup + args.steps + 2)
    s = sess[0]
    occ, K = s["occ"], s["K"]
    H, W = occ.shape
    cores = cprop.host_cores()
    budget = args.ref_budget_s
    f = cprop.Filter(occ[(H - 8) // 2:(H - 8) // 2 + 8], K, s["cell"], threads=cores)
    t1 = time.perf_counter()
    f.step(*s["odom"][0])
    per_cell = (time.perf_counter() - t1) / (8 * W * K)
    rows = int(max(8, min(H, budget / (args.steps + args.warmup) / max(per_cell * W * K, 1e-12))))
    j0 = (H - rows) // 2
    f = cprop.Filter(occ[j0:j0 + rows], K, s["cell"], threads=cores)
    ts = []
    for t in range(args.warmup + args.steps):
        t1 = time.perf_counter()
        f.step(*s["odom"][t])
        ts.append(time.perf_counter() - t1)
    timed = ts[args.warmup:]
    sec = statistics.mean(timed)
    value = rows * W * K / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(wl, sess, ws),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"FP64 oracle step (propagation restated in C, {cores} threads) on a {rows}-row "
                                   f"band of session 0 ({H} x {W}, K = {K}), {len(timed)} timed steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def dense_scans(wl, occ, walk, n):
    """n scans along the walk (poses 1 .. n)."""
    from synth import scan
    return [scan.simulate_scan(occ, wl["cell"], walk.poses[1 + t], seed=wl["seed"] * 97 + t,
                               n_beams=wl["n_beams"], angle_min=wl["angle_min"], angle_inc=wl["angle_inc"],
                               r_max=wl["r_max"], noise_sigma=wl["scan_noise"], dropout=wl["dropout"],
                               march=0.25) for t in range(n)]


def oracle_dense_rate(wl, occ, walk, budget_s: float, steps: int):
    """The oracle's dense scan update on a band of map rows (all bins; the band's own table).
    Returns (state-updates/s, rows, timed steps, seconds per step)."""
    from oracle import dense as D
    from oracle import filter as F
    H, W, K, A = wl["H"], wl["W"], wl["K"], wl["n_angles"]
    z = dense_scans(wl, occ, walk, 1)[0]

    def timed(rows, n):
        j0 = (H - rows) // 2
        band = occ[j0:j0 + rows]
        table = D.range_table(band, A, wl["r_max"], wl["cell"])
        b = F.uniform_belief(F.traversability(band), K)
        ts = []
        for _ in range(n):
            t = time.perf_counter()
            b, _, _, _ = D.dense_update(b, band, table, 0.0, z, wl["angle_min"], wl["angle_inc"], wl["r_max"],
                                        wl["beam_stride"], wl["sigma_r"])
            ts.append(time.perf_counter() - t)
        return ts

    probe = min(H, 8)
    per_row = statistics.mean(timed(probe, 1)) / probe
    rows = int(max(4, min(H, budget_s / max(steps, 1) / max(per_row, 1e-9))))
    ts = timed(rows, steps)
    per = statistics.mean(ts)
    return rows * W * K / per, rows, len(ts), per


def run_dense(args, wl, occ, walk, ws, rank, local):
    """One dense scan update per step (timed), with an odometry step between scans (untimed)."""
    import torch

    import paper_1910_00572_gb300 as loc
    from paper_1910_00572_gb300 import build
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    storage = wl["storage"]
    K, A = wl["K"], wl["n_angles"]
    p = loc.loc_params_default(H=wl["H"], W=wl["W"], K=K, cell_m=wl["cell"], sigma_xy_cells=wl["sigma_xy_cells"],
                               sigma_theta_bins=wl["sigma_theta_bins"], storage=storage, stream=loc.torch_stream())
    h = loc.loc_create(occ, p)
    n_scans = 16
    scans = dense_scans(wl, occ, walk, n_scans)
    n_used = statistics.mean(float((z[::wl["beam_stride"]] < wl["r_max"]).sum()) for z in scans)
    odom = walk.odom
    n_states = wl["H"] * wl["W"] * K
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    scan_args = (wl["angle_min"], wl["angle_inc"], wl["beam_stride"], wl["sigma_r"])
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loc.loc_range_table(h, A, wl["r_max"])
        table_s = time.perf_counter() - t0
        for s in range(args.warmup):
            loc.loc_step(h, *odom[s % len(odom)])
            loc.loc_lidar_update_dense(h, scans[s % n_scans], *scan_args)
        torch.cuda.synchronize()
        barrier(ws)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        with ClockSampler(None) as clk:
            for s in range(args.steps):
                loc.loc_step(h, *odom[(args.warmup + s) % len(odom)])
                flush.zero_()
                starts[s].record()
                loc.loc_lidar_update_dense(h, scans[(args.warmup + s) % n_scans], *scan_args)
                ends[s].record()
            torch.cuda.synchronize()
        barrier(ws)
        ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        total_s = max_over_ranks(sum(ms) / 1e3, ws)
        per_step_s = total_s / args.steps
        # end to end: the scan from host memory in, the pose estimate out
        n_e2e = 0 if args.no_e2e else min(args.steps, 200)
        e2e_t = 0.0
        for s in range(n_e2e):
            loc.loc_step(h, *odom[s % len(odom)])
            torch.cuda.synchronize()
            t = time.perf_counter()
            loc.loc_lidar_update_dense(h, scans[s % n_scans], *scan_args)
            loc.loc_argmax(h)
            e2e_t += time.perf_counter() - t
        e2e_t = max_over_ranks(e2e_t, ws)
        # map difficulty (Eq. 11) on 64 seeded free probe cells, heading bin 0, every 4th direction
        free = np.flatnonzero(occ.reshape(-1) == 0)
        probes = np.random.default_rng(wl["seed"] + 5).choice(free, 64, replace=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dm_err, dm_wrong = loc.loc_map_difficulty(h, probes, 0, 4, wl["sigma_r"], 1.0)
        dm_s = time.perf_counter() - t0
    finally:
        loc.loc_destroy(h)
    if rank != 0:
        return
    flops_state = 3.0 * n_used                    # per used beam: z - q, then (.)^2 accumulated (FMA)
    achieved = n_states * flops_state / (statistics.mean(ms) / 1e3) / 1e12
    peak = 152 * 128 * 2 * 2.070e9 / 1e12
    elem = ELEM[storage]
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        rate, rows, n, per = oracle_dense_rate(wl, occ, walk, 15.0, 2)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"FP64 oracle dense_update on a {rows}-row band ({rows} x {wl['W']} x {K} states, "
                         f"the band's own table), mean of {n} updates, {per:.2f} s each"}
    line = {
        "metric": METRIC, "value": n_states * ws / per_step_s, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": storage, "data": "synthetic",
        "config": config_of(wl, args, extra={"n_angles": A, "r_max": wl["r_max"], "n_beams": wl["n_beams"],
                                             "beam_stride": wl["beam_stride"], "used_beams_mean": n_used,
                                             "timed": "loc_lidar_update_dense (score + reweight of every state)",
                                             "table_build_s": table_s}),
        "p50_step_ms": float(np.percentile(ms, 50)), "p99_step_ms": float(np.percentile(ms, 99)),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "dense_score + dense_apply",
                     "algorithmic_flops_per_launch": n_states * flops_state,
                     "hbm_bytes_per_launch": n_states * (A / K + 8 + 3 * elem),
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"},
        "cpu_baseline": cpu,
        "e2e": {"value": n_states * ws * n_e2e / e2e_t if n_e2e else None, "unit": UNIT,
                "h2d_bytes_per_step": 4 * wl["n_beams"], "d2h_bytes_per_step": 12, "steps": n_e2e,
                "path": "loc_lidar_update_dense (ranges from host memory) + loc_argmax, host wall clock"},
        "gpu_launches": 2 * args.steps,
        "clocks": clk.summary(),
        "map_difficulty": {"probes": int(probes.size), "n_wrong": int(dm_wrong),
                           "D_M": dm_wrong / probes.size, "median_error_m": float(np.median(dm_err)),
                           "ms_per_probe": dm_s * 1e3 / probes.size,
                           "note": "Eq. 11 with C = 1 m on seeded free probe cells (noise-free table scans)"},
    }
    print(json.dumps(line), flush=True)


def run_reference_dense(args, wl, occ, walk, ws, rank):
    if rank != 0:
        return
    rate, rows, n, per = oracle_dense_rate(wl, occ, walk, 150.0, args.steps + args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(wl, args, extra={"sample": f"oracle dense update on a {rows}-row band"}),
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"FP64 oracle dense_update on {rows} x {wl['W']} x {wl['K']} states, {n} updates"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.steps is None:
        args.steps = {"serve256": 60, "office2048_scans": 200}.get(args.workload, 2000)
    ws, rank, local = dist_init(args.gpus)
    wl = workloads.get("office2048" if args.workload == "office2048_scans" else args.workload)
    if args.storage:
        wl["storage"] = args.storage
    if args.workload == "serve256":
        if args.impl == "reference":
            run_reference_serve(args, wl, ws, rank)
        else:
            run_headline(args, wl, ws, rank, local)
    elif args.workload == "office2048_scans":
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable":
                                  "the oracle arm is timed on the single-session and served workloads"}), flush=True)
        else:
            run_office2048_scans(args, ws, rank, local)
    elif args.workload == "batch64":
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable":
                                  "the oracle arm is timed on the single-session and served workloads"}), flush=True)
        else:
            run_batch64(args, wl, ws, rank, local)
    else:
        occ = workloads.make_map(wl)
        walk = workloads.make_walk(wl, occ, seed_offset=rank)
        dense = "n_angles" in wl
        if args.impl == "reference":
            (run_reference_dense if dense else run_reference)(args, wl, occ, walk, ws, rank)
        elif dense:
            run_dense(args, wl, occ, walk, ws, rank, local)
        else:
            run_ours(args, wl, occ, walk, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

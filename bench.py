"""Benchmark: Larger-than-Life steps on GB300 through the cat C ABI.

Workload (default): the radius sweep -- one 16384 x 16384 uint8 grid,
Bernoulli(0.5), zero halo, for every r = 1..16 the radius-scaled rule
R_r C2 M1 S round(0.34n)..round(0.58n) B round(0.34n)..round(0.45n) NM.
One bench step = one LTL step of each of the 16 grids (16 kernel launches,
16 x 2^28 cell updates).  The grids (256 MiB each) exceed the 129 MB L2, so no
flush is needed between launches.

Prints ONE JSON line (metric cell-updates/s).  `--impl reference` times the
CPU oracle (the paper has no code to run) on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-updates/s vs r=1..16: FP8/INT8 batched vs FP16 CAT on GB300, bit-exact"
N = 16384
RADII = list(range(1, 17))
SEED = 2024
P_ALIVE = 0.5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cat", choices=["cat", "reference"])
    ap.add_argument("--dtype", default="fp8", choices=["fp8", "fp16"])
    ap.add_argument("--size", type=int, default=N)
    ap.add_argument("--no-compare", action="store_true", help="skip the comparator kernels")
    ap.add_argument("--cpu-sample", type=int, default=8192,
                    help="rows of the full-width band of the grid the oracle is timed on")
    ap.add_argument("--radii", default="1-16", help="radii to run, e.g. 1-16 or 16 or 1,8,16")
    ap.add_argument("--batch-count", type=int, default=4096, help="grids in the batched workload (0: skip it)")
    ap.add_argument("--multistate-size", type=int, default=49152, help="side of the multi-state grid (0: skip it)")
    ap.add_argument("--no-periodic", action="store_true", help="skip the periodic-boundary measurement")
    ap.add_argument("--no-bits", action="store_true", help="skip the one-bit-storage measurement")
    ap.add_argument("--no-vn", action="store_true", help="skip the simplified von Neumann measurement")
    ap.add_argument("--no-multistep", action="store_true", help="skip the several-steps-per-launch measurement")
    ap.add_argument("--no-wide", action="store_true", help="skip the r > 16 measurement")
    ap.add_argument("--no-fp4", action="store_true", help="skip the FP4 / FP8 precision measurement")
    return ap.parse_args()


def job_rate(ms_total_local, cells_per_step_per_rank, steps, world, dist=None, device="cpu"):
    """Whole-job throughput of `world` replicas: the slowest rank's time over
    `steps` steps, and every rank's cells.  Returns (ms per step, cells/s)."""
    import torch
    ms = float(ms_total_local)
    if world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / steps
    return ms_per_step, cells_per_step_per_rank * world / (ms_per_step / 1000.0)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in ("cat_tc.cu", "ptx.cuh", "cat_internal.h"):
        with open(os.path.join(ROOT, "paper_2406_17284_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, cells: int):
    """DRAM bytes per launch from the committed ncu capture of `kernel` ("fp8", "fp16",
    "vn", "bits"; profiles/traffic.json), scaled to `cells`; None when the kernel source
    changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)
        if rec.get("kernel_source_sha") != kernel_source_sha():
            return None
        cap = rec["captures"][kernel]
        grid = cap.get("grid", rec.get("grid"))
        return cap["traffic_bytes_per_launch"] * cells / (grid[0] * grid[1])
    except Exception:
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# Algorithmic tensor work per cell update: the paper's own granularity, six
# 16x16x16 MMAs per 16x16 fragment of cells (Sec. IV, Alg. 1), 192 flops per
# cell for every r <= 16.  What a kernel executes beyond that is overhead.
FLOPS_PER_CELL = 192.0


def executed_flops_per_cell(short_window: bool) -> float:
    """Tensor flops the tcgen05 Moore kernel issues per cell update, from its
    instruction shapes: pass 1 M = 128, N = 160 (144 in the short window),
    K = 160 and pass 2 M = N = 128, K = 160 per 128 x 128 tile."""
    n1 = 144 if short_window else 160
    return (2 * 128 * n1 * 160 + 2 * 128 * 128 * 160) / (128 * 128)


def measure_tensor_peaks(torch, cat, stream):
    """Dense tcgen05 MMA rates of this GPU (cat_tensor_probe: one CTA per SM issuing
    M=128 N=256 MMAs back to back): burst = median of ten ~2 ms launches,
    sustained = one launch of ~1 s.  TFLOP/s per operand dtype."""
    sms = torch.cuda.get_device_properties(stream.device).multi_processor_count
    status = torch.zeros(1, dtype=torch.int32, device=stream.device)
    out = {}
    for name, dt, K in (("e4m3", cat.DTYPE_FP8_E4M3, 32), ("e2m1", cat.DTYPE_FP4_E2M1, 32), ("f16", cat.DTYPE_FP16, 16)):
        def flops(n):
            return sms * n * 2.0 * 128 * 256 * K
        n_burst, n_sus = 1 << 15, 1 << 23
        for _ in range(3):
            cat.cat_tensor_probe(dt, n_burst, status.data_ptr(), stream)
        t = time_launches(torch, lambda: cat.cat_tensor_probe(dt, n_burst, status.data_ptr(), stream), 10, stream)
        burst = flops(n_burst) / (statistics.median(t) / 1000.0) / 1e12
        t = time_launches(torch, lambda: cat.cat_tensor_probe(dt, n_sus, status.data_ptr(), stream), 1, stream)
        sustained = flops(n_sus) / (t[0] / 1000.0) / 1e12
        torch.cuda.synchronize()
        if int(status.item()) != 0:
            raise RuntimeError(f"tensor probe ({name}) timed out")
        out[name] = {"burst_tflops": burst, "sustained_tflops": sustained}
    out["how"] = ("cat_tensor_probe: one CTA per SM, one thread issuing tcgen05.mma M=128 N=256 (K=32 e4m3 or e2m1 "
                  "kind::f8f6f4 / K=16 f16 kind::f16), f32 accumulators; burst = median of 10 launches of "
                  "2^15 MMAs per SM, sustained = one launch of 2^23")
    return out


def roof(value, bytes_per_cell, tensor_tflops, hbm_gbs, tensor_src="e4m3 burst"):
    """The roofline of a path in cell-updates/s: the slower of the HBM term (state
    bytes per cell update at the measured copy rate) and the tensor term (192
    flops per cell update at the operand dtype's measured dense rate; None where
    the path does not run on tcgen05), and value's fraction of it."""
    hbm_term = hbm_gbs * 1e9 / bytes_per_cell
    tensor_term = tensor_tflops * 1e12 / FLOPS_PER_CELL if tensor_tflops else None
    bound = "tensor" if tensor_term is not None and tensor_term < hbm_term else "hbm"
    rl = min(hbm_term, tensor_term) if tensor_term is not None else hbm_term
    return {"bound": bound, "roofline_cell_updates_per_s": rl, "frac": value / rl,
            "hbm_term": hbm_term, "tensor_term": tensor_term, "bytes_per_cell": bytes_per_cell,
            "tensor_peak": tensor_src if tensor_term is not None else None}


def host_link(torch, dev, nbytes=256 << 20, reps=5):
    """Plain pinned-memory copies of nbytes: host->device, device->host, and both at
    once on two streams (GB/s, median of reps, CUDA events)."""
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h2 = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    d2 = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    out = {}
    for name, fn in (("h2d_gbs", lambda: d.copy_(h, non_blocking=True)),
                     ("d2h_gbs", lambda: h.copy_(d, non_blocking=True))):
        with torch.cuda.stream(s1):
            fn()
            t = time_launches(torch, fn, reps, s1)
        out[name] = nbytes / (statistics.median(t) / 1000.0) / 1e9
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s1):
            d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    out["bidirectional_gbs_each_way"] = nbytes / statistics.median(ts) / 1e9
    out["bytes"] = nbytes
    return out


# ------------------------------------------------------------- CPU oracle
def oracle_sample(rows: int, radii, steps: int = 1, width: int = N):
    """Times the oracle (as it stands) on the first `rows` full-width rows of the
    workload's grid, one step per radius."""
    from oracle import oracle
    from paper_2406_17284_gb300 import inputs
    grid = inputs.bernoulli_window(N, N, P_ALIVE, SEED, 0, 0, rows, width)
    lib = oracle.load()
    t0 = time.perf_counter()
    for r in radii:
        rule = oracle.Rule(**inputs.scaled_rule(r, M=1))
        oracle.step(grid, rule, n_steps=steps, lib=lib)
    dt = time.perf_counter() - t0
    cells = rows * width * len(radii) * steps
    return cells / dt, dt, oracle.num_threads(lib)


def run_reference(args, rank, world):
    if rank != 0:
        return
    side = max(64, args.cpu_sample // 4)   # bounded per-step sample: the whole run stays within minutes
    vals = []
    for _ in range(max(1, args.warmup)):
        oracle_sample(min(side, 256), RADII[:2])
    t_all = 0.0
    for _ in range(args.steps):
        v, dt, cores = oracle_sample(side, RADII)
        vals.append(v)
        t_all += dt
    value = statistics.median(vals)
    # measured wall time of one reference step: one step per radius of the
    # sampled band (side rows x N columns), not a projection to the full grid
    ms_per_step = 1000.0 * t_all / args.steps
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": f"radius_sweep_{N}x{N}_r1-16_bernoulli0.5", "grid": [N, N], "radii": RADII,
                   "rule": "R_r C2 M1 S0.34n..0.58n B0.34n..0.45n NM", "boundary": "zero",
                   "l2": "inputs larger than L2"},
        "step": f"one step per r in {RADII[0]}..{RADII[-1]} of the first {side} rows x {N} columns "
                f"({side * N * len(RADII)} cell updates, measured)",
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {side} rows x {N} columns of the 16384^2 grid, one step per r in {RADII[0]}..{RADII[-1]}"},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- GPU arm
def time_launches(torch, fn, reps, stream):
    """Average device time of fn() (one or more launches) with CUDA events on `stream`."""
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def measure_batch(args, torch, cat, inputs, stream, steps_per_graph=64):
    """The heterogeneous batch: `count` grids (sides log-uniform in [64, 2048], r uniform
    in 1..16, M uniform in {0,1}, p uniform in [0.2, 0.6], the scaled rule, C = 2), 64
    steps per CUDA-graph launch.  FP8 and FP16 tcgen05 batched launches, and the
    paper-style FP16 mma.sync kernel launched per grid, on the same states."""
    from oracle import oracle
    specs = inputs.batch_instances(args.batch_count, seed=SEED)
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(min(32, os.cpu_count() or 1)) as ex:
        hosts = list(ex.map(lambda d: inputs.bernoulli(d["H"], d["W"], d["p"], d["seed"]), specs))
    cells = sum(h.size for h in hosts)
    grids = [cat.Grid(d["H"], d["W"], d["rule"], kernel="tcgen05", dtype="fp8") for d in specs]
    for g, h in zip(grids, hosts):
        cat.cat_set_state(g.handle, h.ctypes.data, h.shape[1], False, stream)
    stream.synchronize()
    handles = [g.handle for g in grids]
    out = {"workload": f"{args.batch_count} grids, sides log-uniform in [64, 2048] (independent H, W), "
                       "r uniform 1..16, M uniform {0,1}, p uniform [0.2, 0.6], scaled rule C2",
           "cells": int(cells), "steps_per_launch_graph": steps_per_graph}
    done = 0

    def timed(fn, reps):
        evs = time_launches(torch, fn, reps, stream)
        return statistics.median(evs)

    # FP8 tcgen05, one persistent launch per step, 64 steps per graph
    cat.cat_batch_step(handles, steps_per_graph, stream)   # plan + graph built, warm-up
    done += steps_per_graph
    ms = timed(lambda: cat.cat_batch_step(handles, steps_per_graph, stream), 3)
    done += 3 * steps_per_graph
    out["fp8_tcgen05_batched"] = cells * steps_per_graph / (ms / 1000.0)
    # bit-exactness of the 8 smallest grids after all steps so far
    small = sorted(range(len(specs)), key=lambda i: hosts[i].size)[:8]
    stream.synchronize()
    for i in small:
        want = oracle.step(hosts[i], oracle.Rule(**specs[i]["rule"]), n_steps=done)
        if not np.array_equal(grids[i].get_state(stream), want):
            raise RuntimeError(f"batched grid {i} differs from the oracle")
    out["oracle_checked_grids"] = len(small)
    # FP16 tcgen05 batched
    for g in grids:
        cat.cat_set_options(g.handle, cat.KERNEL_TCGEN05, cat.DTYPE_FP16)
    cat.cat_batch_step(handles, steps_per_graph, stream)
    ms = timed(lambda: cat.cat_batch_step(handles, steps_per_graph, stream), 2)
    out["fp16_tcgen05_batched"] = cells * steps_per_graph / (ms / 1000.0)
    # the paper's FP16 fragment scheme, one launch per grid and step
    for g in grids:
        cat.cat_set_options(g.handle, cat.KERNEL_MMA_SYNC, cat.DTYPE_FP16)
    cat.cat_batch_step(handles, 1, stream)
    ms = timed(lambda: cat.cat_batch_step(handles, 4, stream), 1)
    out["fp16_paper_mma_sync_per_grid"] = cells * 4 / (ms / 1000.0)
    for g in grids:
        g.close()
    return out


def measure_multistate(args, torch, cat, inputs, stream):
    """The multi-state workload: a 49152^2 grid with states uniform over {0..15} under
    R10 C16 M1 S150..260 B150..200 (FP8 operands, window re-encoded so only state 1
    counts), timed over its first steps while it still holds decaying cells, and a
    batch of 256 such grids of 2048^2."""
    rule = inputs.MULTISTATE_R10_C16
    n = args.multistate_size
    out = {"workload": f"{n}x{n} and 256 x 2048x2048, states uniform over 0..15, R10 C16 M1 S150..260 B150..200"}
    init = inputs.uniform_states(n, n, 16, 4915)
    g = cat.Grid(n, n, rule, kernel="tcgen05", dtype="fp8")
    g.set_state(init)
    g.step(1, stream)
    t = time_launches(torch, lambda: g.step(1, stream), 4, stream)
    out["single_cell_updates_per_s"] = n * n / (statistics.median(t) / 1000.0)
    g.close()
    # the same grid stored four bits per cell (1 byte of state traffic per update),
    # on the operands CAT_DTYPE_AUTO takes there
    g = cat.Grid(n, n, rule, kernel="tcgen05", dtype="auto", storage=cat.STORE_NIB4)
    out["single_nib4_dtype"] = {v: k for k, v in cat.DTYPES.items()}[cat.cat_get_options(g.handle)["dtype"]]
    g.set_state(init)
    g.step(1, stream)
    t = time_launches(torch, lambda: g.step(1, stream), 4, stream)
    out["single_nib4_cell_updates_per_s"] = n * n / (statistics.median(t) / 1000.0)
    g.close()
    del init
    grids = [cat.Grid(2048, 2048, rule, kernel="tcgen05", dtype="fp8") for _ in range(256)]
    for i, gg in enumerate(grids):
        gg.set_state(inputs.uniform_states(2048, 2048, 16, 5000 + i))
    handles = [gg.handle for gg in grids]
    cat.cat_batch_step(handles, 4, stream)                  # plan + graph built
    ms = statistics.median(time_launches(torch, lambda: cat.cat_batch_step(handles, 4, stream), 3, stream))
    out["batch_256x2048_cell_updates_per_s"] = 256 * 2048 * 2048 * 4 / (ms / 1000.0)
    for gg in grids:
        gg.close()
    return out


def measure_periodic(args, torch, cat, inputs, stream, radii=(1, 8, 16)):
    """The same 16384^2 Bernoulli(0.5) grid and scaled rules with the periodic
    boundary (each step = ghost-frame refresh + tcgen05 step), FP8 operands."""
    n = args.size
    init = inputs.bernoulli(n, n, 0.5, SEED)
    out = {"workload": f"{n}x{n} periodic, scaled rule C2 M1, fp8"}
    for r in radii:
        g = cat.Grid(n, n, inputs.scaled_rule(r, M=1), kernel="tcgen05", dtype="fp8", boundary=cat.BOUNDARY_PERIODIC)
        g.set_state(init)
        g.step(1, stream)
        t = time_launches(torch, lambda: g.step(1, stream), 3, stream)
        out[f"r{r}_cell_updates_per_s"] = n * n / (statistics.median(t) / 1000.0)
        g.close()
    return out


def measure_sweep(torch, cat, stream, grids, n, reps=3):
    """Median device time per launch (ms) of each grid's step, the grids stepped
    round-robin (radius order) reps times after one warm-up round."""
    for r in RADII:
        grids[r].step(1, stream)
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in RADII]
           for _ in range(reps)]
    for row in evs:
        for (a, b), r in zip(row, RADII):
            a.record(stream)
            grids[r].step(1, stream)
            b.record(stream)
    torch.cuda.synchronize()
    per_r = {r: statistics.median(row[i][0].elapsed_time(row[i][1]) for row in evs) for i, r in enumerate(RADII)}
    for g in grids.values():
        assert g.status() == cat.CAT_OK
        g.close()
    return per_r


def measure_vn(args, torch, cat, inputs, stream, d_init, hbm):
    """Simplified von Neumann neighbourhood (Eq. 3): the headline's 16384^2 grid with
    the cross-scaled rules (n = 4r + 1, C2 M1), FP8 operands, uint8 storage (2 bytes
    of algorithmic traffic per cell update), stepped round-robin over the radii."""
    n = args.size
    grids = {r: cat.Grid(n, n, inputs.vn_scaled_rule(r, M=1), kernel="tcgen05", dtype="fp8") for r in RADII}
    for g in grids.values():
        g.set_state(d_init)
    per_r = measure_sweep(torch, cat, stream, grids, n)
    ms = sum(per_r.values())
    achieved = 2.0 * n * n * len(RADII) / (ms / 1000.0) / 1e9
    paper = {}   # the paper-style FP16 fragment kernel on the same grid (Eq. 3 as printed)
    if not args.no_compare:
        for r in (1, 8, 16):
            g = cat.Grid(n, n, inputs.vn_scaled_rule(r, M=1), kernel="mma_sync", dtype="fp16")
            g.set_state(d_init)
            g.step(1, stream)
            t = time_launches(torch, lambda: g.step(1, stream), 3, stream)
            paper[str(r)] = n * n / (statistics.median(t) / 1000.0)
            g.close()
    return {"workload": f"radius_sweep_{n}x{n}_r1-16_bernoulli0.5, simplified von Neumann, fp8",
            "paper_fp16_fragments_cell_updates_per_s": paper,
            "cell_updates_per_s": n * n * len(RADII) / (ms / 1000.0),
            "per_r_cell_updates_per_s": {str(r): n * n / (t / 1000.0) for r, t in per_r.items()},
            "bytes_per_cell": 2.0, "achieved_gbs": achieved, "hbm_frac": achieved / hbm,
            "traffic_bytes_per_launch": recorded_traffic("vn", n * n), "kernel": "ltl_vn_kernel"}


def measure_multistep(torch, cat, inputs, stream, steps=64):
    """Small single grids (L2-resident), the scaled rule r = 4 (FP8): `steps` steps with
    one launch per step (cat_step, k = 1) and with all of them in one cooperative
    launch (k = steps, CTAs meeting on a grid barrier between steps); and one-bit
    grids under Conway's rule on the bit-sliced kernel, one launch per step
    against 8 steps per launch (temporal blocking)."""
    out = {"workload": f"{steps} steps of one grid, scaled rule r=4 C2 M1, fp8"}
    for n in (512, 1024, 2048):
        init = torch.from_numpy(inputs.bernoulli(n, n, 0.5, SEED + n)).cuda()
        for k in (1, steps):
            g = cat.Grid(n, n, inputs.scaled_rule(4, M=1), kernel="tcgen05", dtype="fp8", steps_per_launch=k)
            g.set_state(init)
            g.step(steps, stream)
            t = time_launches(torch, lambda: g.step(steps, stream), 3, stream)
            assert g.status() == cat.CAT_OK
            out[f"{n}x{n}_k{k}_cell_updates_per_s"] = n * n * steps / (statistics.median(t) / 1000.0)
            g.close()
    # temporal blocking of the bit-sliced kernel on one-bit grids, Conway's rule
    # (r = 1): one launch per step against 8 steps per launch on tiles kept in
    # shared memory
    for n in (512, 2048, 16384):
        init = torch.from_numpy(inputs.bernoulli(n, n, 0.5, SEED + n)).cuda()
        for k in (1, 8):
            g = cat.Grid(n, n, inputs.CONWAY, kernel="bitslice", storage=cat.STORE_BIT1, steps_per_launch=k)
            g.set_state(init)
            g.step(steps, stream)
            t = time_launches(torch, lambda: g.step(steps, stream), 3, stream)
            assert g.status() == cat.CAT_OK
            out[f"bits_conway_{n}x{n}_k{k}_cell_updates_per_s"] = n * n * steps / (statistics.median(t) / 1000.0)
            g.close()
    return out


def measure_wide(args, torch, cat, inputs, stream, d_init):
    """Radii beyond 16 on the headline's grid: the tcgen05 kernel on 128 x 128 tiles in
    a 192 x 192 window (32-cell halo, e4m3 digits against a band of ones and a band of
    16s, f32 pass 2; the default), the same on 96 x 96 tiles in a 160 x 160 window, and
    the FP16 fragment kernel with a second halo fragment (five band fragments per
    reduction, FP32 step-2 accumulation)."""
    n = args.size
    out = {"workload": f"{n}x{n} bernoulli0.5, scaled rule C2 M1, r > 16: tcgen05 (fp8) on 128x128 tiles in a "
                       "192-row window and on 96x96 tiles, and the FP16 fragment kernel", "kernel": "ltl_big_kernel"}
    for kern, dt, key, kw in (("tcgen05", "fp8", "tcgen05_fp8", {}), ("tcgen05", "fp8", "tcgen05_fp8_tile96", dict(tile=96)),
                              ("mma_sync", "fp16", "fragment_fp16", {})):
        for r in (17, 24, 32):
            g = cat.Grid(n, n, inputs.scaled_rule(r, M=1), kernel=kern, dtype=dt, **kw)
            g.set_state(d_init)
            g.step(1, stream)
            t = time_launches(torch, lambda: g.step(1, stream), 3, stream)
            assert g.status() == cat.CAT_OK
            out[f"{key}_r{r}_cell_updates_per_s"] = n * n / (statistics.median(t) / 1000.0)
            g.close()
    return out


def measure_bits(args, torch, cat, inputs, stream, d_init, hbm):
    """One-bit storage: the headline's 16384^2 grid and 16 scaled rules stored 8 cells
    per byte (FP8 operands), stepped round-robin over the radii like the headline, so
    16 x 64 MiB pass between two steps of one grid (more than L2).  The algorithmic
    traffic is 1/8 byte read + 1/8 byte written per cell update."""
    n = args.size
    grids = {r: cat.Grid(n, n, inputs.scaled_rule(r, M=1), kernel="tcgen05", dtype="fp8", storage=cat.STORE_BIT1)
             for r in RADII}
    for g in grids.values():
        g.set_state(d_init)
    per_r = measure_sweep(torch, cat, stream, grids, n)
    ms = sum(per_r.values())
    achieved = 0.25 * n * n * len(RADII) / (ms / 1000.0) / 1e9
    # the bit-sliced CUDA-core kernel on the same packed grids, r <= 5
    sliced = {}
    for r in [r for r in RADII if r <= 5]:
        g = cat.Grid(n, n, inputs.scaled_rule(r, M=1), kernel="bitslice", storage=cat.STORE_BIT1)
        g.set_state(d_init)
        g.step(2, stream)
        t = time_launches(torch, lambda: g.step(1, stream), 5, stream)
        assert g.status() == cat.CAT_OK
        sliced[str(r)] = n * n / (statistics.median(t) / 1000.0)
        g.close()
    return {"workload": f"radius_sweep_{n}x{n}_r1-16_bernoulli0.5, one bit per cell, fp8",
            "cell_updates_per_s": n * n * len(RADII) / (ms / 1000.0),
            "per_r_cell_updates_per_s": {str(r): n * n / (t / 1000.0) for r, t in per_r.items()},
            "bitslice_cell_updates_per_s": sliced,
            "bytes_per_cell": 0.25, "achieved_gbs": achieved, "hbm_frac": achieved / hbm,
            "traffic_bytes_per_launch": recorded_traffic("bits", n * n), "kernel": "ltl_bits_kernel"}


PREC_N, PREC_P, PREC_RADII = 32768, 0.35, (1, 5, 10, 16)


def measure_fp4(args, torch, cat, inputs, stream):
    """Operand precisions on tcgen05 at the precision workload's size (32768^2,
    Bernoulli(0.35), the scaled rule C2 M1, r in {1, 5, 10, 16}): FP4 (e2m1
    pass-1 operands, e4m3 digits in pass 2) and FP8 (e4m3) on uint8, one-bit and
    four-bit storage, the median of five launches per grid."""
    n = PREC_N if args.size == N else args.size
    init = torch.from_numpy(inputs.bernoulli(n, n, PREC_P, SEED + 3)).to(stream.device)
    out = {"workload": f"{n}x{n} bernoulli{PREC_P}, scaled rule C2 M1, r in {list(PREC_RADII)}",
           "bytes_per_cell": {"u8": 2.0, "bit1": 0.25, "nib4": 1.0}}
    for st_name, st in (("u8", cat.STORE_U8), ("bit1", cat.STORE_BIT1), ("nib4", cat.STORE_NIB4)):
        for dt in ("fp4", "fp8"):
            row = {}
            for r in PREC_RADII:
                g = cat.Grid(n, n, inputs.scaled_rule(r, M=1), kernel="tcgen05", dtype=dt, storage=st)
                g.set_state(init)
                g.step(2, stream)
                t = time_launches(torch, lambda: g.step(1, stream), 5, stream)
                assert g.status() == cat.CAT_OK
                row[str(r)] = n * n / (statistics.median(t) / 1000.0)
                g.close()
            out[f"{dt}_{st_name}_cell_updates_per_s"] = row
    del init
    torch.cuda.empty_cache()
    return out


def run_cat(args, rank, world, local):
    import torch
    import torch.distributed as dist

    from paper_2406_17284_gb300 import build as cat_build
    from paper_2406_17284_gb300 import cat, inputs

    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    cat_build.build()
    cat.load()
    n = args.size
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    tensor_peaks = measure_tensor_peaks(torch, cat, stream)
    e4m3_peak = tensor_peaks["e4m3"]["burst_tflops"]
    f16_peak = tensor_peaks["f16"]["burst_tflops"]
    host = inputs.bernoulli(n, n, P_ALIVE, SEED + rank)
    d_init = torch.from_numpy(host).to(dev)
    grids = {}
    for r in RADII:
        g = cat.Grid(n, n, inputs.scaled_rule(r, M=1), kernel="tcgen05", dtype=args.dtype)
        g.set_state(d_init)
        grids[r] = g
    torch.cuda.synchronize()

    # the radii grouped by the kernel instantiation that serves them (with FP8
    # operands the short-window kernel r <= 7, the standard one r >= 8); a step
    # launches one group after the other, so CUDA events at the group
    # boundaries time each kernel live inside the timed region while the
    # launches of a group run back to back (each may start while the previous
    # one drains: programmatic dependent launch)
    kern_of = {r: ("ltl_tc_kernel<FP8, short window>" if args.dtype == "fp8" and r <= 7
                   else f"ltl_tc_kernel<{args.dtype.upper()}, standard window>") for r in RADII}
    groups = {}
    for r in RADII:
        groups.setdefault(kern_of[r], []).append(r)

    def one_step():
        for rs in groups.values():
            for r in rs:
                grids[r].step(1, stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        per_group = []
        t0.record(stream)
        for _ in range(args.steps):
            for kname, rs in groups.items():
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for r in rs:
                    grids[r].step(1, stream)
                b.record(stream)
                per_group.append((kname, len(rs), a, b))
        t1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    for g in grids.values():
        rc = g.status()
        if rc != cat.CAT_OK:
            raise RuntimeError(f"device status {rc}")
    cells_per_step = n * n * len(RADII)
    ms_per_step, value = job_rate(t0.elapsed_time(t1), cells_per_step, args.steps, world, dist, dev)
    group_ms = {}
    for kname, cnt, a, b in per_group:
        group_ms.setdefault(kname, []).append(a.elapsed_time(b) / cnt)
    kernel_launch_ms = {k: statistics.mean(v) for k, v in group_ms.items()}   # average launch, live
    avg_launch_ms = sum(kernel_launch_ms[kern_of[r]] for r in RADII) / len(RADII)
    # per radius (after the timed region): each launch between its own events,
    # behind one untimed launch so that the first event is not recorded on an
    # idle device ahead of the host's launch call
    per_r = {}
    for r in RADII:
        grids[r].step(1, stream)
        t = time_launches(torch, lambda: grids[r].step(1, stream), 3, stream)
        per_r[r] = statistics.mean(t)

    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    alg_bytes = 2.0 * n * n  # read + write of one uint8 state per cell
    achieved_all = alg_bytes / (avg_launch_ms / 1000.0) / 1e9
    # the dominant kernel: the instantiation with the larger share of the
    # timed region's launch time (its average launch from the group events)
    share = {k: kernel_launch_ms[k] * len(rs) for k, rs in groups.items()}
    dom = max(share, key=share.get)
    dom_ms = kernel_launch_ms[dom]
    achieved = alg_bytes / (dom_ms / 1000.0) / 1e9
    tpeak = e4m3_peak if args.dtype == "fp8" else f16_peak
    dom_roof = roof(n * n / (dom_ms / 1000.0), 2.0, tpeak, hbm)

    # ---- e2e: same metric through the C ABI from pinned host memory.  Every
    # step of every grid copies its input in (cat_set_state), steps it and
    # copies the result out (cat_get_state), on three streams so that the
    # host-to-device copy of one grid, the step of another and the
    # device-to-host copy of a third overlap (a grid's next input waits for
    # its previous result to be read out; results alternate between two
    # pinned buffers).
    pin_in = torch.from_numpy(host).pin_memory()
    pin_out = [torch.empty_like(pin_in).pin_memory() for _ in range(2)]
    # (the host link's rate varies between runs: the best of three runs of up
    # to three steps each is reported)
    e2e_steps, e2e_runs = max(1, min(args.steps, 3)), 3
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    te_runs = []
    for _ in range(e2e_runs):
        read_out = {r: None for r in RADII}
        torch.cuda.synchronize()
        te0 = time.perf_counter()
        k = 0
        for _ in range(e2e_steps):
            for r in RADII:
                g = grids[r]
                if read_out[r] is not None:
                    s_in.wait_event(read_out[r])
                cat.cat_set_state(g.handle, pin_in.data_ptr(), n, False, s_in)
                copied = torch.cuda.Event()
                copied.record(s_in)
                stream.wait_event(copied)
                g.step(1, stream)
                stepped = torch.cuda.Event()
                stepped.record(stream)
                s_out.wait_event(stepped)
                cat.cat_get_state(g.handle, pin_out[k & 1].data_ptr(), n, False, s_out)
                k += 1
                read_out[r] = torch.cuda.Event()
                read_out[r].record(s_out)
        torch.cuda.synchronize()
        te_runs.append((time.perf_counter() - te0) / e2e_steps)
    te = min(te_runs)
    e2e_value = cells_per_step * world / te

    link = host_link(torch, dev)

    # ---- comparators on the same inputs (median of a few launches per r)
    comps = {}
    if not args.no_compare and rank == 0:
        variants = [("tcgen05", "fp16" if args.dtype == "fp8" else "fp8"), ("mma_sync", "fp16"),
                    ("mma_sync", "int8"), ("stencil", "auto"), ("runsum", "auto")]
        for kern, dt in variants:
            row = {}
            for r in RADII:
                g = cat.Grid(n, n, inputs.scaled_rule(r, M=1), kernel=kern, dtype=dt)
                g.set_state(d_init)
                reps = 3 if kern != "stencil" else 2
                g.step(1, stream)
                t = time_launches(torch, lambda: g.step(1, stream), reps, stream)
                row[r] = n * n / (statistics.median(t) / 1000.0)
                g.close()
            comps[f"{kern}/{dt}"] = row

    batched = None
    if args.batch_count > 0 and rank == 0:
        batched = measure_batch(args, torch, cat, inputs, stream)
    multistate = None
    if args.multistate_size > 0 and rank == 0:
        multistate = measure_multistate(args, torch, cat, inputs, stream)
    periodic = None
    if not args.no_periodic and rank == 0:
        periodic = measure_periodic(args, torch, cat, inputs, stream)
    bits = None
    if not args.no_bits and rank == 0:
        bits = measure_bits(args, torch, cat, inputs, stream, d_init, hbm)
    vn = None
    if not args.no_vn and rank == 0:
        vn = measure_vn(args, torch, cat, inputs, stream, d_init, hbm)
    multistep = None
    if not args.no_multistep and rank == 0:
        multistep = measure_multistep(torch, cat, inputs, stream)
    wide = None
    if not args.no_wide and rank == 0:
        wide = measure_wide(args, torch, cat, inputs, stream, d_init)
    fp4 = None
    if not args.no_fp4 and rank == 0:
        fp4 = measure_fp4(args, torch, cat, inputs, stream)

    cpu = None
    if rank == 0:
        v, dt, cores = oracle_sample(args.cpu_sample, RADII)
        cpu = {"value": v, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
               "sample": f"first {args.cpu_sample} rows x {N} columns of the grid, one step per r in {RADII[0]}..{RADII[-1]} ({dt:.1f} s)"}

    for g in grids.values():
        g.close()

    # every figure next to its own roofline (state bytes per cell update; the
    # tensor term where the path runs on tcgen05, at that operand dtype's rate)
    def roofs(d, keys, bpc, tflops):
        if d is not None:
            d["roofline"] = {k: roof(d[k], bpc, tflops, hbm) for k in keys if d.get(k)}
    if batched:
        roofs(batched, ["fp8_tcgen05_batched"], 2.0, e4m3_peak)
        batched["roofline"].update({k: roof(batched[k], 2.0, f16_peak, hbm, "f16 burst")
                                    for k in ["fp16_tcgen05_batched"] if batched.get(k)})
        batched["roofline"].update({k: roof(batched[k], 2.0, None, hbm)
                                    for k in ["fp16_paper_mma_sync_per_grid"] if batched.get(k)})
    roofs(multistate, ["single_cell_updates_per_s", "batch_256x2048_cell_updates_per_s"], 2.0, e4m3_peak)
    if multistate and multistate.get("single_nib4_cell_updates_per_s"):
        multistate["roofline"]["single_nib4_cell_updates_per_s"] = roof(
            multistate["single_nib4_cell_updates_per_s"], 1.0, e4m3_peak, hbm)
    roofs(periodic, [k for k in (periodic or {}) if k.endswith("_per_s")], 2.0, e4m3_peak)
    roofs(bits, ["cell_updates_per_s"], 0.25, e4m3_peak)
    if bits and bits.get("bitslice_cell_updates_per_s"):   # CUDA cores: the one-bit HBM term
        bits["bitslice_roofline"] = {r: roof(v, 0.25, None, hbm) for r, v in bits["bitslice_cell_updates_per_s"].items()}
    roofs(vn, ["cell_updates_per_s"], 2.0, e4m3_peak)
    roofs(multistep, [k for k in (multistep or {}) if k.endswith("_per_s") and not k.startswith("bits_")], 2.0, e4m3_peak)
    if multistep:
        multistep["roofline"].update({k: roof(v, 0.25, None, hbm) for k, v in multistep.items()
                                      if k.startswith("bits_") and k.endswith("_per_s")})
    roofs(wide, [k for k in (wide or {}) if k.endswith("_per_s")], 2.0, None)
    if fp4:   # per storage and dtype: that storage's bytes, that operand dtype's tensor rate
        e2m1_peak = tensor_peaks["e2m1"]["burst_tflops"]
        fp4["roofline_frac"] = {
            k: {r: roof(v, fp4["bytes_per_cell"][k.split("_")[1]], e2m1_peak if k.startswith("fp4") else e4m3_peak,
                        hbm, "e2m1 burst" if k.startswith("fp4") else "e4m3 burst")["frac"] for r, v in row.items()}
            for k, row in fp4.items() if k.endswith("_per_s")}
    comp_roofs = {}
    for k, row in comps.items():
        tp = f16_peak if k == "tcgen05/fp16" else e4m3_peak if k == "tcgen05/fp8" else None
        comp_roofs[k] = {str(r): roof(v, 2.0, tp, hbm)["frac"] for r, v in row.items()}
    if rank == 0:
        per_r_rate = {str(r): n * n / (ms / 1000.0) for r, ms in sorted(per_r.items())}
        line = {
            "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "e4m3" if args.dtype == "fp8" else "f16",
            "dtype_detail": ("e4m3" if args.dtype == "fp8" else "f16") + " operands, f16 accumulators (exact), u8 states",
            "data": "synthetic",
            "config": {"workload": f"radius_sweep_{n}x{n}_r1-16_bernoulli0.5", "grid": [n, n], "radii": RADII,
                       "rule": "R_r C2 M1 S0.34n..0.58n B0.34n..0.45n NM", "boundary": "zero",
                       "kernel": f"tcgen05/{args.dtype}", "l2": "inputs (256 MiB per grid) larger than L2",
                       "parallelism": f"replicas x{world}"},
            "gpu_launches": args.steps * len(RADII),
            "roofline": {"bound": dom_roof["bound"], "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": recorded_traffic(args.dtype, n * n),
                         "peak_source": f"{peak_kind} hbm_gbs (burst copy)", "kernel": dom,
                         "kernel_radii": [r for r in RADII if kern_of[r] == dom],
                         "launch_time_source": "CUDA events around each step's back-to-back launches of this kernel "
                                               "in the timed region, divided by their count",
                         "kernel_time_share": share[dom] / sum(share.values()),
                         "hbm_term_cell_updates_per_s": dom_roof["hbm_term"],
                         "tensor_term_cell_updates_per_s": dom_roof["tensor_term"],
                         "executed_flops_per_cell": executed_flops_per_cell("short" in dom),
                         "executed_tflops": n * n / (dom_ms / 1000.0) * executed_flops_per_cell("short" in dom) / 1e12,
                         "executed_frac_of_tensor_peak": n * n / (dom_ms / 1000.0) * executed_flops_per_cell("short" in dom)
                                                         / (tpeak * 1e12),
                         "tensor_term": f"{FLOPS_PER_CELL:.0f} flops per cell update at the measured "
                                        f"{'e4m3' if args.dtype == 'fp8' else 'f16'} burst rate {tpeak:.0f} TFLOP/s",
                         "all_radii": {"achieved": achieved_all, "frac": achieved_all / hbm}},
            "tensor_peaks_tflops": tensor_peaks,
            "roofline_whole_sweep": roof(value / world, 2.0, tpeak, hbm),
            "per_r_cell_updates_per_s": per_r_rate,
            "per_r_source": "after the timed region: one untimed launch, then three launches per radius, each between its own CUDA events",
            "comparators_cell_updates_per_s": {k: {str(r): v for r, v in row.items()} for k, row in comps.items()},
            "comparators_roofline_frac": comp_roofs,
            # the headline kernel's rate over the fastest CUDA-core kernel (direct
            # stencil or separable running sums) at each r
            "tensor_core_over_best_cuda_core": {
                str(r): per_r_rate[str(r)] / max(comps[k][r] for k in ("stencil/auto", "runsum/auto") if k in comps)
                for r in RADII} if "runsum/auto" in comps else None,
            "batched": batched,
            "multistate": multistate,
            "periodic": periodic,
            "bits": bits,
            "von_neumann": vn,
            "multistep": multistep,
            "wide_radius": wide,
            "precisions": fp4,
            "e2e": {"value": e2e_value, "unit": "cell-updates/s", "h2d_bytes_per_step": n * n * len(RADII),
                    "runs_cell_updates_per_s": [cells_per_step * world / t for t in te_runs],
                    "method": f"best of {e2e_runs} runs of {e2e_steps} steps",
                    "d2h_bytes_per_step": n * n * len(RADII), "host_link": link,
                    "link_bound_cell_updates_per_s": link["bidirectional_gbs_each_way"] * 1e9 * world},
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def parse_radii(spec: str):
    out = []
    for part in spec.split(","):
        if "-" in part:
            a, b = part.split("-")
            out += list(range(int(a), int(b) + 1))
        else:
            out.append(int(part))
    assert all(1 <= r <= 16 for r in out)
    return out


def main():
    global RADII
    args = parse()
    RADII = parse_radii(args.radii)
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_cat(args, rank, world, local)


if __name__ == "__main__":
    main()

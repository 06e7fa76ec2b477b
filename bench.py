"""Throughput of batched local-GP distance-field inference on GB300.

Default workload (the large G-GPDF query): a 100x100x10 m synthetic city (ground + 200 boxes),
2,000,000 surface points, 10,000,000 query points (70 % uniform in free space, 30 % within
0.5 m of a surface), 27-leaf neighbourhoods capped at 1024 points, l = 0.3 m, sigma = 0.01.
One step = bin the surface into leaves (vgp_set_surface) + one G-GPDF distance+gradient query
of all 10M points (vgp_query_distance_gradient), mixed precision (FP32 kernel values / mean /
gradient, FP64 Cholesky, solves and reverting).  ``value`` is queries per second with inputs
resident in HBM; ``e2e`` is the same through the C ABI with the inputs copied from pinned host
memory and the results copied back inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "G-GPDF distance+gradient queries/sec and L-GPDF voxels/sec vs FP64 plain, at stated error"
UNIT = "queries/s"
WORKLOAD = "city G-GPDF: 2M surface pts, 10M queries (70% free space, 30% <=0.5 m from surface), 27-leaf cap 1024"


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _scene(rank: int, n_surface: int, n_query: int):
    from paper_2407_09649_gb300 import scenes
    city = scenes.City(0)
    S = city.surface(n=n_surface, seed=0)
    Q = city.queries(n=n_query, seed=1 + rank)
    return S, Q


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except FileNotFoundError:
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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


# FP64 pipe of GB300 from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP64_ALU_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2407_09649_gb300 import _lib
    from paper_2407_09649_gb300.api import Map

    ws, rank, local = _dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    S_h, Q_h = _scene(rank, args.n_surface, args.n_query)
    S = torch.from_numpy(S_h).to(dev)
    Q = torch.from_numpy(Q_h).to(dev)
    nq = Q.shape[0]
    m = Map(precision="mixed", profile=0)
    out = {"d": torch.empty(nq, dtype=torch.float64, device=dev),
           "grad": torch.empty((nq, 3), dtype=torch.float64, device=dev),
           "status": torch.empty(nq, dtype=torch.uint8, device=dev)}
    lib = _lib.load()

    def step():
        m.set_surface(S)
        m.query(Q, grad=True, var=False, out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    l0 = lib.vgp_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(args.steps):
            step()
        ev1.record()
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = int(lib.vgp_launch_count() - l0)
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    value = ws * nq * args.steps / (ms / 1e3)
    st = m.stats()

    # the dominant kernel (GP solve: Cholesky + alpha + evaluation), timed with events
    mp = Map(precision="mixed", profile=1)
    mp.set_surface(S)
    mp.query(Q, grad=True, var=False, out=out)
    sp = mp.stats()
    solve_ms = sp["t_solve_ms"]
    fp64_flops = sp["sum_n3"] / 3.0 + 2.0 * sp["sum_n2"]
    achieved = fp64_flops / (solve_ms / 1e3) / 1e12

    extra = {}
    if not args.quick:
        # variance on (extra FP64 triangular solve per query)
        outv = dict(out, var=torch.empty(nq, dtype=torch.float64, device=dev))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        m.set_surface(S)
        m.query(Q, grad=True, var=True, out=outv)
        b.record()
        torch.cuda.synchronize()
        extra["variance_on_queries_per_s"] = nq / (a.elapsed_time(b) / 1e3)
        # plain FP64 (batched)
        m64 = Map(precision="fp64")
        m64.set_surface(S)
        m64.query(Q, grad=True, var=False, out=out)
        torch.cuda.synchronize()
        a.record()
        m64.set_surface(S)
        m64.query(Q, grad=True, var=False, out=out)
        b.record()
        torch.cuda.synchronize()
        extra["fp64_batched_queries_per_s"] = nq / (a.elapsed_time(b) / 1e3)

    # end to end through the C ABI: pinned host inputs in, results out, every step
    S_pin = torch.from_numpy(S_h).pin_memory()
    Q_pin = torch.from_numpy(Q_h).pin_memory()
    d_pin = torch.empty(nq, dtype=torch.float64).pin_memory()
    g_pin = torch.empty((nq, 3), dtype=torch.float64).pin_memory()
    S_d = torch.empty_like(S)
    Q_d = torch.empty_like(Q)

    def e2e_step():
        S_d.copy_(S_pin, non_blocking=True)
        Q_d.copy_(Q_pin, non_blocking=True)
        m.set_surface(S_d)
        m.query(Q_d, grad=True, var=False, out=out)
        d_pin.copy_(out["d"], non_blocking=True)
        g_pin.copy_(out["grad"], non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e_steps = max(1, min(args.steps, 3))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(e_steps):
        e2e_step()
    b.record()
    torch.cuda.synchronize()
    e_ms = a.elapsed_time(b) / e_steps
    if ws > 1:
        t = torch.tensor([e_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e_ms = float(t.item())

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(S_h, Q_h, args.cpu_sample)

    if rank == 0:
        pk = _peaks()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic (seeded city scene)",
            "config": {"workload": WORKLOAD, "n_surface": int(S.shape[0]), "n_queries": int(nq),
                       "precision": "mixed (FP32 eval, FP64 factorisation/solves/reverting)",
                       "variance": False, "l2": "inputs+outputs (~460 MB) larger than L2",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "instances": st["n_instances"], "query_leaves": st["n_groups"],
                       "bucket_count": st["bucket_count"]},
            "e2e": {"value": ws * nq / (e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": int(S_h.nbytes + Q_h.nbytes), "d2h_bytes_per_step": int(nq * 32)},
            "gpu_launches": launches,
            "roofline": {"kernel": "k_solve (K assembly, FP64 Cholesky, alpha, fused eval)", "bound": "alu",
                         "pipe": "fp64", "achieved": achieved, "peak": FP64_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_ALU_PEAK_TFLOPS, "traffic": None,
                         "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz",
                         "solve_ms": solve_ms, "algorithmic_fp64_flop": fp64_flops},
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        line.update(extra)
        if pk:
            line["peaks_file"] = {k: pk.get(k) for k in ("hbm_gbs", "bf16_tflops")}
        print(json.dumps(line))
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def cpu_baseline(S_h, Q_h, n_sample):
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    q = Q_h[:n_sample]
    t0 = time.perf_counter()
    surf = oracle.Surface(S_h, oracle.params())
    surf.query(q, want_var=False)
    dt = time.perf_counter() - t0
    return {"value": len(q) / dt, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"first {len(q)} of the 10M queries against the full 2M-point surface (surface binning included)",
            "seconds": dt}


def run_reference(args):
    ws, rank, local = _dist_env()
    if rank != 0:
        return
    S_h, Q_h = _scene(0, args.n_surface, args.n_query)
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    n = args.ref_sample
    times = []
    for i in range(args.warmup + args.steps):
        q = Q_h[i * n:(i + 1) * n]
        t0 = time.perf_counter()
        surf = oracle.Surface(S_h, oracle.params())
        surf.query(q, want_var=False)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    value = n / float(np.mean(times))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded city scene)",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "n_surface": int(S_h.shape[0]), "n_queries": int(Q_h.shape[0]),
                       "precision": "fp64 oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": f"{n} queries per step against the full 2M-point surface"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-surface", type=int, default=2_000_000)
    ap.add_argument("--n-query", type=int, default=10_000_000)
    ap.add_argument("--cpu-sample", type=int, default=2000)
    ap.add_argument("--ref-sample", type=int, default=1000)
    ap.add_argument("--quick", action="store_true", help="skip the variance-on and FP64 comparison lines")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

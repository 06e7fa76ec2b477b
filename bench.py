"""Throughput of batched local-GP distance-field inference on GB300.

Default workload (the large G-GPDF query): a 100x100x10 m synthetic city (ground + 200 boxes),
2,000,000 surface points, 10,000,000 query points (70 % uniform in free space, 30 % within
0.5 m of a surface), 27-leaf neighbourhoods capped at 1024 points, l = 0.3 m, sigma = 0.01.
One step = bin the surface into leaves (vgp_set_surface) + one G-GPDF distance+gradient query
of all 10M points (vgp_query_distance_gradient), mixed precision (FP32 kernel values / mean /
gradient; FP64-accurate Cholesky whose large trailing updates run as exact integer-slice
products on the bf16 tensor cores; FP64 solves and reverting).  ``value`` is queries per
second with inputs resident in HBM, timed without any instrumentation; ``e2e`` is the same
through the C ABI with the inputs copied from pinned host memory and the results copied back
inside the timed region.  Kernel times for the roofline lines come from a separate pass of
the same configuration with the library's profile mode (CUDA events on the launching stream).

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

# DRAM bytes (read + write) of the N > 224 solve launch (k_solve_emu) of one full 10M-query
# step: 708.2 GB from an ncu capture of the current kernel on the 100k-query city case, scaled
# by the ratio of the two launches' algorithmic work (sum of N^3/3 + 2 N^2: 2.854e12 against
# 1.851e12 flop, x1.542; an earlier kernel's small and full-size captures had that ratio).
# None when the kernel has changed since.
K_SOLVE_TRAFFIC = 1.0921e12
K_SOLVE_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the N > 224 launch (k_solve_emu) on "
                          "the 100k-query city case, scaled to the full step by its algorithmic work; "
                          "smaller buckets not included")

# Algorithmic DRAM bytes of the HBM-bound steps (what each step must move at least):
#   bin (S1): read the point (12 B) and write its leaf slot (4 B); the leaf table and its
#             counters stay in L2
#   gather (S3): read each candidate's index and point (4 + 12 B), write each kept training
#             point in FP64 and FP32 with its global index (24 + 12 + 8 B), 24 B of centre per
#             instance
#   fuse (S9): read key, d, v, status of a testing voxel (25 B), read and write D and V (32 B)
BIN_BYTES_PER_POINT = 16
GATHER_BYTES_PER_CAND, GATHER_BYTES_PER_POINT, GATHER_BYTES_PER_INST = 16, 44, 24
FUSE_BYTES_PER_VOXEL = 57


def _dist_env():
    from paper_2407_09649_gb300 import replicas
    return replicas.rank_env()


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


def bf16_peak_tflops(pk):
    """Measured dense bf16 burst peak (MEASURED_PEAKS.json), else the recipe's fallback."""
    return float(pk.get("bf16_tflops") or 1900.0)


# FP64 tensor path (mma.sync m8n8k4 f64) peak: the measured bf16 dense peak times the nominal
# FP64 / bf16 ratio of GB300 (1.25 / 2250 TFLOP/s).
def fp64_tensor_peak_tflops(pk):
    return bf16_peak_tflops(pk) * 1.25 / 2250.0


def hbm_peak_gbs(pk):
    return float(pk.get("hbm_gbs") or 6800.0)


def _emu_mma_table():
    """bf16 tensor flops of the emulated factorisation of one instance, by N (0..1024).

    The factorisation runs in blocks of 4 tiles (32 columns); after each block but the last,
    the M = Nt - K1 row tiles below it take a trailing update in bands of 16 row tiles (128
    rows); a band meets ceil((b0 + nb) / 4) column tiles of 32 columns (b0: the band's first
    row tile, nb its row tiles), and each (band, column tile) output is 2 steps x 34 slice
    products of tcgen05.mma kind::f16 M = 128, N = 32, K = 16 (2 * 128 * 32 * 16 flops each)."""
    tab = np.zeros(1025)
    for N in range(1, 1025):
        Nt = (N + 7) // 8
        mmas = 0
        for K0 in range(0, Nt, 4):
            K1 = min(K0 + 4, Nt)
            if K1 >= Nt:
                break
            M = Nt - K1
            for b0 in range(0, M, 16):
                nb = min(16, M - b0)
                mmas += ((b0 + nb + 3) // 4) * 2 * 34
        tab[N] = mmas * (2 * 128 * 32 * 16)
    return tab


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2407_09649_gb300 import _lib, replicas
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
    # emulate_fp64=1: the trailing Cholesky updates of the N > 32 instances run as exact
    # integer-slice products on the bf16 tensor cores, recombined to FP64 accuracy; profile off
    m = Map(precision="mixed", emulate_fp64=1)
    out = {"d": torch.empty(nq, dtype=torch.float64, device=dev),
           "grad": torch.empty((nq, 3), dtype=torch.float64, device=dev),
           "status": torch.empty(nq, dtype=torch.uint8, device=dev)}
    lib = _lib.load()

    def step():
        m.set_surface(S)
        m.query(Q, grad=True, var=False, out=out)

    # launch shapes per size bucket from the library's autotuner, on a query subset
    m.set_surface(S)
    tuned = m.autotune(Q[: min(nq, args.n_tune)].contiguous())

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
    value, sec = replicas.aggregate(nq * args.steps, ms / 1e3, ws, device=dev)
    ms_step = sec * 1e3 / args.steps
    st = m.stats()

    # the same configuration instrumented (profile mode: CUDA events on the launching stream
    # around the solve, bin and gather kernels), outside the timed region
    prof = instrumented_pass(Map, S, Q, out, tuned, args.prof_steps)

    extra = {}
    if not args.quick and rank == 0:
        extra = comparisons(S, Q, S_h, Q_h, args)

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
    e_value, _ = replicas.aggregate(nq * e_steps, a.elapsed_time(b) / 1e3, ws, device=dev)

    cpu = None
    err = None
    if rank == 0 and not args.no_cpu:
        # the CPU-baseline leg: the oracle's G-GPDF sample, the error against it, and its frame
        cpu = cpu_baseline(S_h, Q_h, args.cpu_sample, args.cpu_sample_1t)
        err = error_vs_oracle(S_h, Q_h, m, args.cpu_sample)
        if "lgpdf_sphere_plane" in extra:
            extra["lgpdf_sphere_plane"]["oracle"] = oracle_frame_baseline()

    if rank == 0:
        pk = _peaks()
        peak = fp64_tensor_peak_tflops(pk)
        bf16_peak = bf16_peak_tflops(pk)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64+bf16", "data": "synthetic (seeded city scene)",
            "config": {"workload": WORKLOAD, "n_surface": int(S.shape[0]), "n_queries": int(nq),
                       "precision": ("mixed: FP32 kernel values, mean and gradient; FP64 panels, diagonal "
                                     "blocks, solves and reverting; for N > 32 instances float-pair K entries "
                                     "(FP32 pipe) and the Cholesky trailing updates as exact bf16 slice "
                                     "products on the tensor cores (FP32 accumulation, integer recombination "
                                     "into a 2^-61 fixed-point trailing matrix); FP64 K entries below"),
                       "variance": False, "l2": "inputs+outputs (~460 MB) larger than L2",
                       "instrumentation": "none in the timed steps (kernel times from a separate profile pass)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "instances": st["n_instances"], "query_leaves": st["n_groups"],
                       "bucket_count": st["bucket_count"], "autotuned_launch": tuned},
            "e2e": {"value": e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(S_h.nbytes + Q_h.nbytes), "d2h_bytes_per_step": int(nq * 32)},
            "gpu_launches": launches,
            "roofline": solve_roofline(prof, peak, bf16_peak),
            "hbm_kernels": hbm_lines(prof, extra.pop("_fuse_prof", None), hbm_peak_gbs(pk)),
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "error_vs_oracle": err,
        }
        line.update(extra)
        if pk:
            line["peaks_file"] = {k: pk.get(k) for k in ("hbm_gbs", "bf16_tflops")}
        print(json.dumps(line))
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def instrumented_pass(Map, S, Q, out, tuned, steps):
    """The headline configuration with profile = 1 (CUDA events around the solve launches of
    each call, and around the bin and gather kernels), over ``steps`` full steps after one
    warm-up step; the N distribution comes from the query plan of the same queries."""
    import torch
    mp = Map(precision="mixed", emulate_fp64=1, profile=1)
    mp.set_launch(tuned["threads"], tuned["per_sm"], tuned["stage_panel"])
    acc = {"solve_ms": 0.0, "emu_ms": 0.0, "bin_ms": 0.0, "gather_ms": 0.0, "cand": 0, "train": 0, "inst": 0,
           "points": 0, "sum_n3": 0.0, "sum_n2": 0.0}
    for it in range(steps + 1):
        mp.set_surface(S)
        sb = mp.stats()
        mp.query(Q, grad=True, var=False, out=out)
        sq = mp.stats()
        if it == 0:
            continue
        acc["bin_ms"] += sb["t_bin_ms"]
        acc["points"] += sb["n_points"]
        acc["solve_ms"] += sq["t_solve_ms"]
        acc["emu_ms"] += sum(sq["t_bucket_ms"][:4])  # the emulated launches: N > 32
        acc["gather_ms"] += sq["t_gather_ms"]
        acc["cand"] += sq["n_candidates"]
        acc["train"] += sq["n_train"]
        acc["inst"] += sq["n_instances"]
        acc["sum_n3"] += sq["sum_n3"]
        acc["sum_n2"] += sq["sum_n2"]
    torch.cuda.synchronize()
    plan = mp.debug_query_plan(Q)
    N = np.diff(plan["inst_off"])
    acc = {k: v / steps for k, v in acc.items()}
    acc["N"] = N
    mp.close()
    return acc


def solve_roofline(prof, fp64_peak, bf16_peak):
    """The dominant kernel: the GP solve launches (k_solve_emu for N > 32, k_solve below).
    FP64-equivalent Cholesky work over the solve time against the FP64 tensor peak, and the
    bf16 slice products actually issued by k_solve_emu over its own time against the bf16
    peak."""
    N = prof["N"]
    flop = prof["sum_n3"] / 3.0 + 2.0 * prof["sum_n2"]
    achieved = flop / (prof["solve_ms"] / 1e3) / 1e12
    big = N[N > 32].astype(np.int64)
    bf16_flop = float(_emu_mma_table()[big].sum())
    bf16_achieved = bf16_flop / (prof["emu_ms"] / 1e3) / 1e12 if prof["emu_ms"] > 0 else None
    return {"kernel": ("k_solve_emu (N > 32: FP64-accurate Cholesky, trailing updates as bf16 slice products) + "
                       "k_solve (N <= 32: FP64 tile Cholesky on mma.sync f64); alpha, fused eval"),
            "bound": "tensor", "dtype": "fp64 (FP64-equivalent work)", "achieved": achieved, "peak": fp64_peak,
            "unit": "TFLOP/s", "frac": achieved / fp64_peak,
            "frac_note": ("achieved counts the FP64 Cholesky flops the method needs; the emulated updates run "
                          "them on the bf16 pipe, so frac exceeds 1 against the FP64 tensor peak; bf16_pipe "
                          "gives the fraction of the pipe that executes them"),
            "traffic": K_SOLVE_TRAFFIC, "traffic_source": K_SOLVE_TRAFFIC_SOURCE,
            "peak_source": "of measured: MEASURED_PEAKS bf16_tflops x nominal FP64/bf16 (1.25/2250)",
            "solve_ms": prof["solve_ms"], "algorithmic_fp64_flop": flop,
            "algorithmic_flop_def": "sum over instances of N^3/3 + 2 N^2",
            "bf16_pipe": {"kernel": "k_solve_emu", "achieved": bf16_achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                          "frac": bf16_achieved / bf16_peak if bf16_achieved else None,
                          "peak_source": "of measured: MEASURED_PEAKS bf16_tflops (cuBLAS burst)",
                          "kernel_ms": prof["emu_ms"], "bf16_flop": bf16_flop,
                          "flop_def": ("tcgen05.mma kind::f16 128x32x16 slice products issued: per 32-column "
                                       "block, per band of 128 rows, ceil(rows reached / 32) column tiles x 2 steps "
                                       "x 34 products x 131072 flop")}}


def hbm_lines(prof, fuse_prof, peak):
    """HBM roofline fractions of the bin (S1), gather (S3) and fuse (S9) kernels from their
    profile-mode CUDA-event times and the algorithmic bytes above."""
    out = {}
    if prof["bin_ms"] > 0:
        by = BIN_BYTES_PER_POINT * prof["points"]
        gbs = by / (prof["bin_ms"] / 1e3) / 1e9
        out["bin"] = {"kernel": "k_surface_bin", "bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                      "frac": gbs / peak, "kernel_ms": prof["bin_ms"], "bytes": by,
                      "bytes_def": f"{BIN_BYTES_PER_POINT} B per surface point", "units": prof["points"]}
    if prof["gather_ms"] > 0:
        by = (GATHER_BYTES_PER_CAND * prof["cand"] + GATHER_BYTES_PER_POINT * prof["train"]
              + GATHER_BYTES_PER_INST * prof["inst"])
        gbs = by / (prof["gather_ms"] / 1e3) / 1e9
        out["gather"] = {"kernel": "k_inst_gather", "bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "kernel_ms": prof["gather_ms"], "bytes": by,
                         "bytes_def": (f"{GATHER_BYTES_PER_CAND} B per candidate + {GATHER_BYTES_PER_POINT} B per "
                                       f"training point + {GATHER_BYTES_PER_INST} B per instance"),
                         "candidates": prof["cand"], "training_points": prof["train"], "instances": prof["inst"]}
    if fuse_prof and fuse_prof["ms"] > 0:
        by = FUSE_BYTES_PER_VOXEL * fuse_prof["voxels"]
        gbs = by / (fuse_prof["ms"] / 1e3) / 1e9
        out["fuse"] = {"kernel": "k_fuse_insert + k_fuse_alloc + k_fuse_update", "bound": "hbm", "achieved": gbs,
                       "peak": peak, "unit": "GB/s", "frac": gbs / peak, "kernel_ms": fuse_prof["ms"], "bytes": by,
                       "bytes_def": f"{FUSE_BYTES_PER_VOXEL} B per testing voxel",
                       "workload": fuse_prof["workload"]}
    out["peak_source"] = "of measured: MEASURED_PEAKS hbm_gbs (copy)"
    return out


def _timed(fn, reps=1):
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps / 1e3


def comparisons(S, Q, S_h, Q_h, args):
    """Secondary lines, each timed with CUDA events after a warm-up call."""
    out = {}
    out.update(city_lines(S, Q, args))
    out.update(sphere_plane_lines(args))
    out.update(room_lines(args))
    out.update(sweep_lines(args))
    return out


def city_lines(S, Q, args):
    """On the city workload: the all-FP64 tensor path, variance on (full size), the precision
    subset, the blended Eq. 10 G-GPDF, and the plain FP64 per-instance form."""
    from paper_2407_09649_gb300.api import Map
    out = {}
    # the headline workload with every Cholesky update on the FP64 tensor path (no emulation)
    mpl = Map(precision="mixed", profile=1)
    mpl.set_surface(S)
    mpl.autotune(Q[: min(Q.shape[0], args.n_tune)].contiguous())
    acc = {"ms": 0.0, "flop": 0.0}

    def plain_step():
        mpl.set_surface(S)
        mpl.query(Q, grad=True, var=False)
        sp = mpl.stats()
        acc["ms"] += sp["t_solve_ms"]
        acc["flop"] += sp["sum_n3"] / 3.0 + 2.0 * sp["sum_n2"]

    t = _timed(plain_step, reps=2)  # one warm-up call, then two timed; acc is a ratio over all three
    tf = acc["flop"] / (acc["ms"] / 1e3) / 1e12
    out["plain_fp64_tensor_path"] = {"queries": int(Q.shape[0]), "queries_per_s": Q.shape[0] / t,
                                     "ms_per_step": 1e3 * t, "k_solve_tflops": tf,
                                     "frac_of_fp64_peak": tf / fp64_tensor_peak_tflops(_peaks()),
                                     "note": "profile mode on (per-bucket events)"}
    mpl.close()
    # variance on, all 10M queries, the headline map
    mv = Map(precision="mixed", emulate_fp64=1)
    mv.set_surface(S)
    t = _timed(lambda: (mv.set_surface(S), mv.query(Q, grad=True, var=True)))
    out["variance_on_full"] = {"queries": int(Q.shape[0]), "queries_per_s": Q.shape[0] / t, "ms_per_step": 1e3 * t,
                               "precision": "mixed, emulate_fp64=1, FP64 variance solve"}
    mv.close()
    nsub = min(args.n_sub, Q.shape[0])
    Qs = Q[:nsub].contiguous()
    res = {}
    for name, kw, var in (("mixed", dict(precision="mixed"), False), ("mixed_var", dict(precision="mixed"), True),
                          ("fp64", dict(precision="fp64"), False), ("fp64_var", dict(precision="fp64"), True)):
        m = Map(**kw)
        t = _timed(lambda: (m.set_surface(S), m.query(Qs, grad=True, var=var)))
        res[name] = nsub / t
    out["subset_queries"] = nsub
    out["subset_queries_per_s"] = res
    # G-GPDF as blended per-leaf GPs (Eq. 10, 8 nodes, lambda 100 / m), the full 10M queries
    msm = Map(precision="mixed", max_pts_leaf=512, emulate_fp64=1)
    t = _timed(lambda: (msm.set_surface(S), msm.query_smooth(Q, n_nodes=8, lam=100.0, grad=True)))
    out["smooth_min_8_nodes"] = {"queries": int(Q.shape[0]), "queries_per_s": Q.shape[0] / t,
                                 "leaf_gps": msm.stats()["n_instances"]}
    msm.close()
    # plain FP64 per-instance launches (the comparison form), on a smaller subset
    npi = min(args.n_per_instance, Q.shape[0])
    Qp = Q[:npi].contiguous()
    mp = Map(precision="fp64", launch="per_instance")
    mb = Map(precision="mixed", emulate_fp64=1)
    tp = _timed(lambda: (mp.set_surface(S), mp.query(Qp, grad=True, var=False)))
    tb = _timed(lambda: (mb.set_surface(S), mb.query(Qp, grad=True, var=False)))
    out["per_instance_fp64"] = {"queries": npi, "queries_per_s": npi / tp, "instances": mp.stats()["n_instances"],
                                "batched_mixed_same_queries_per_s": npi / tb, "speedup_batched_mixed": tp / tb}
    return out


def sphere_plane_lines(args):
    """The plain FP64 single frame (20k points on a sphere of radius 2 m and the plane z = -1,
    cap 64 per leaf): L-GPDF build + fuse in testing voxels per second, FP64 and mixed, the
    per-instance FP64 form and the 10k queries (the FP64 oracle on the same frame is timed by
    the CPU-baseline leg, oracle_frame_baseline)."""
    import torch
    from paper_2407_09649_gb300 import scenes
    from paper_2407_09649_gb300.api import Map
    pts = scenes.sphere_plane_frame(0)
    q = scenes.uniform_queries(0)
    pt = torch.from_numpy(pts).cuda()
    qt = torch.from_numpy(q).cuda()
    res = {}
    # mixed: with the emulated updates (instances above 32 points), as the headline map
    for name, kw in (("fp64", dict(precision="fp64")), ("mixed", dict(precision="mixed", emulate_fp64=1)),
                     ("per_instance_fp64", dict(precision="fp64", launch="per_instance"))):
        m = Map(**kw)
        nvox = {}

        def frame():
            f = m.build_frame(pt)
            nvox["n"] = f.n_test
            m.fuse(f)

        t = _timed(frame, reps=args.frame_reps)
        m.set_surface(pt)
        tq = _timed(lambda: m.query(qt, grad=True, var=True), reps=args.frame_reps)
        res[name] = {"voxels_per_s": nvox["n"] / t, "ms_per_frame": 1e3 * t, "testing_voxels": nvox["n"],
                     "queries_per_s": len(q) / tq, "leaf_gps": m.stats()["n_instances"]}
        m.close()
    res["workload"] = ("sphere r=2 m + plane z=-1, 20k points, sigma 0.01 m noise, voxel 0.1 m, cap 64 per leaf; "
                       "testing voxels = all voxels of occupied leaves and their 26 neighbours; 10k uniform queries")
    return {"lgpdf_sphere_plane": res}


def room_lines(args):
    """The room sequence (100k-point frames on a circular camera path, leaf cap 512):
    L-GPDF frames/voxels per second, ray-cast testing points, the whole mapping step, the
    per-instance FP64 form, the fusion kernels' time (profile), and backward throughput of the
    autograd function over the room map (256 trajectories x 64 waypoints)."""
    import torch
    from paper_2407_09649_gb300 import scenes
    from paper_2407_09649_gb300.api import Map
    from paper_2407_09649_gb300.autograd import gpdf_distance
    out = {}
    room = scenes.Room(0)
    frames = [torch.from_numpy(room.frame(k, seed=0)).cuda() for k in range(args.room_frames)]
    poses = [room.camera_pose(k)[0] for k in range(args.room_frames)]

    def run_frames(mr, origin):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nvox = 0
        a.record()
        for fr, o in zip(frames, poses):
            f = mr.build_frame(fr, origin=o if origin else None)
            nvox += f.n_test
            mr.fuse(f)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3, nvox

    for prec in ("mixed", "fp64"):
        # mixed: with the emulated updates (instances above 32 points), as the headline map
        mr = Map(precision=prec, max_pts_leaf=512, emulate_fp64=int(prec == "mixed"))
        mr.fuse(mr.build_frame(frames[0]))
        sec, nvox = run_frames(mr, False)
        out.setdefault("lgpdf_room", {})[prec] = {"voxels_per_s": nvox / sec, "frames": len(frames),
                                                 "emulate_fp64": int(prec == "mixed"),
                                                 "ms_per_frame": 1e3 * sec / len(frames),
                                                 "testing_voxels_per_frame": nvox / len(frames)}
        mr.close()
    # the plain FP64 per-instance form of the L-GPDF (one launch per leaf GP) on two frames
    mq = Map(precision="fp64", max_pts_leaf=512, launch="per_instance")
    mq.fuse(mq.build_frame(frames[0]))
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nvox = 0
    a.record()
    for fr in frames[1:3]:
        f = mq.build_frame(fr)
        nvox += f.n_test
        mq.fuse(f)
    b.record()
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    out["lgpdf_room"]["per_instance_fp64"] = {
        "voxels_per_s": nvox / sec, "frames": 2, "ms_per_frame": 1e3 * sec / 2,
        "speedup_batched_mixed": out["lgpdf_room"]["mixed"]["voxels_per_s"] / (nvox / sec)}
    mq.close()
    # L-GPDF with the paper's testing points: ray-cast from the sensor origin, signed distances
    mr = Map(precision="mixed", max_pts_leaf=512, emulate_fp64=1)
    mr.fuse(mr.build_frame(frames[0], origin=poses[0]))
    sec, nvox = run_frames(mr, True)
    out["lgpdf_room_raycast"] = {"voxels_per_s": nvox / sec, "frames": len(frames),
                                 "ms_per_frame": 1e3 * sec / len(frames),
                                 "testing_voxels_per_frame": nvox / len(frames), "precision": "mixed, emulated updates above 32 points"}
    mr.close()
    # the fusion kernels alone (profile mode), dilated testing sets of all frames
    mf = Map(precision="mixed", max_pts_leaf=512, profile=1)
    mf.fuse(mf.build_frame(frames[0]))
    fms, fvox = 0.0, 0
    for fr in frames:
        f = mf.build_frame(fr)
        fvox += f.n_test
        mf.fuse(f)
        fms += mf.stats()["t_fuse_ms"]
    out["_fuse_prof"] = {"ms": fms, "voxels": fvox,
                         "workload": f"room sequence, {len(frames)} frames, dilated testing voxels"}
    mf.close()
    # whole mapping step per frame: ray-cast L-GPDF, fusion, zero crossings of the touched leaves,
    # G-GPDF retrained on the kept training set; then the marching-cubes mesh of the whole map
    mp = Map(precision="mixed", max_pts_leaf=512, emulate_fp64=1)
    mp.fuse(mp.build_frame(frames[0], origin=poses[0]))
    mp.update_surface()
    torch.cuda.synchronize()
    a.record()
    for fr, o in zip(frames, poses):
        mp.fuse(mp.build_frame(fr, origin=o))
        mp.update_surface()
    b.record()
    torch.cuda.synchronize()
    sec = a.elapsed_time(b) / 1e3
    a.record()
    mesh = mp.extract_mesh(active_only=False, triangles=True)
    b.record()
    torch.cuda.synchronize()
    out["room_mapping_step"] = {"ms_per_frame": 1e3 * sec / len(frames), "frames": len(frames),
                                "training_points": int(mp.surface_points().shape[0]),
                                "mesh_ms": a.elapsed_time(b), "mesh_triangles": int(mesh["triangles"][0].shape[0]),
                                "zero_crossings": int(mesh["crossings"][0].shape[0]), "precision": "mixed, emulated updates above 32 points"}
    surf = mp.surface_points()
    mp.close()
    # the same mapping step with three colour channels per point (Eq. 6 properties, fused)
    mc = Map(precision="mixed", max_pts_leaf=512, n_props=3, emulate_fp64=1)
    cols = [torch.rand((fr.shape[0], 3), device="cuda", generator=torch.Generator("cuda").manual_seed(k))
            for k, fr in enumerate(frames)]
    mc.fuse(mc.build_frame(frames[0], origin=poses[0], props=cols[0]))
    torch.cuda.synchronize()
    a.record()
    for fr, o, col in zip(frames, poses, cols):
        mc.fuse(mc.build_frame(fr, origin=o, props=col))
        mc.update_surface()
    b.record()
    torch.cuda.synchronize()
    out["room_mapping_step_rgb"] = {"ms_per_frame": a.elapsed_time(b) / len(frames), "frames": len(frames),
                                    "n_props": 3, "precision": "mixed, emulated updates above 32 points"}
    mc.close()
    # the same mapping step with every GP solve replayed as a CUDA graph (VGP_LAUNCH_GRAPH)
    mg = Map(precision="mixed", max_pts_leaf=512, launch="graph", emulate_fp64=1)
    mg.fuse(mg.build_frame(frames[0], origin=poses[0]))
    mg.update_surface()
    torch.cuda.synchronize()
    a.record()
    for fr, o in zip(frames, poses):
        mg.fuse(mg.build_frame(fr, origin=o))
        mg.update_surface()
    b.record()
    torch.cuda.synchronize()
    gst = mg.stats()
    out["room_mapping_step_graph"] = {"ms_per_frame": a.elapsed_time(b) / len(frames), "frames": len(frames),
                                      "graph_replays": int(gst["graph_replays"]),
                                      "graph_instantiations": int(gst["graph_instantiations"]),
                                      "precision": "mixed, emulated updates above 32 points"}
    mg.close()
    # differentiation: loss = sum softplus(0.5 m - d) over 256 x 64 waypoints on the room map
    # (the G-GPDF training set the mapping step kept), forward + backward through autograd
    W = torch.from_numpy(room.trajectories(seed=2).reshape(-1, 3)).cuda().requires_grad_(True)
    X = surf.clone().requires_grad_(True)
    mb = Map(precision="fp64")

    def fwd_bwd():
        W.grad = None
        X.grad = None
        d = gpdf_distance(W, X, mb)
        torch.nn.functional.softplus(0.5 - d).sum().backward()

    t = _timed(fwd_bwd, reps=args.frame_reps)
    tf = _timed(lambda: gpdf_distance(W.detach(), X.detach(), mb), reps=args.frame_reps)
    out["backward_room"] = {"waypoints": int(W.shape[0]), "surface_points": int(X.shape[0]),
                            "waypoints_per_s_fwd_bwd": W.shape[0] / t, "ms_fwd_bwd": 1e3 * t, "ms_fwd": 1e3 * tf,
                            "precision": "fp64 (forward and backward)",
                            "map": f"training set kept by the {len(frames)}-frame room mapping step"}
    mb.close()
    return out


def sweep_lines(args):
    """Independent-instance sweep: N log-uniform in [4, 1024], 512 queries each; batched mixed
    (emulated updates) and all-FP64 on all instances, and the plain FP64 per-instance form
    against the batched mixed form on the same subset of instances."""
    import torch
    from paper_2407_09649_gb300 import scenes
    from paper_2407_09649_gb300.api import Map
    out = {}
    io, X, qo, Qw = scenes.patch_sweep(n_inst=args.sweep_inst, seed=4)
    io_d = torch.from_numpy(io).cuda()
    qo_d = torch.from_numpy(qo).cuda()
    X_d = torch.from_numpy(X).cuda()
    Q_d = torch.from_numpy(Qw).cuda()
    for name, kw in (("mixed_emulated", dict(precision="mixed", emulate_fp64=1)), ("fp64", dict(precision="fp64"))):
        mw = Map(**kw)
        t = _timed(lambda: mw.gp_batch(io_d, X_d, qo_d, Q_d, var=False))
        out.setdefault("sweep", {})[name] = {"instances": args.sweep_inst, "queries": int(Qw.shape[0]),
                                             "queries_per_s": Qw.shape[0] / t, "ms": 1e3 * t}
        mw.close()
    del X_d, Q_d
    torch.cuda.empty_cache()
    # per-instance FP64 form on a subset (every k-th instance), against batched mixed on it
    k = max(1, args.sweep_inst // args.sweep_per_instance)
    pick = np.arange(0, args.sweep_inst, k)
    N = np.diff(io)[pick]
    sio = np.concatenate([[0], np.cumsum(N)])
    sX = np.concatenate([X[io[i]:io[i + 1]] for i in pick])
    sQ = np.concatenate([Qw[qo[i]:qo[i + 1]] for i in pick])
    sqo = np.concatenate([[0], np.cumsum(np.diff(qo)[pick])])
    sio, sqo = torch.from_numpy(sio).cuda(), torch.from_numpy(sqo).cuda()
    sX, sQ = torch.from_numpy(sX).cuda(), torch.from_numpy(sQ).cuda()
    mp = Map(precision="fp64", launch="per_instance")
    mb = Map(precision="mixed", emulate_fp64=1)
    tp = _timed(lambda: mp.gp_batch(sio, sX, sqo, sQ, var=False))
    tb = _timed(lambda: mb.gp_batch(sio, sX, sqo, sQ, var=False))
    out["sweep"]["per_instance_fp64_subset"] = {"instances": int(len(pick)), "queries": int(sQ.shape[0]),
                                                "queries_per_s": sQ.shape[0] / tp,
                                                "batched_mixed_same_queries_per_s": sQ.shape[0] / tb,
                                                "speedup_batched_mixed": tp / tb}
    return out


def oracle_frame_baseline():
    """CPU-baseline leg: the FP64 oracle's L-GPDF frame of the sphere + plane scene (testing
    voxels per second, one thread and all host cores)."""
    import oracle
    from paper_2407_09649_gb300 import scenes
    pts = scenes.sphere_plane_frame(0)
    oracle.build()
    cores = os.cpu_count() or 1
    orc = {}
    for th in (1, cores):
        oracle.set_threads(th)
        t0 = time.perf_counter()
        f = oracle.frame(pts, oracle.params())
        dt = time.perf_counter() - t0
        orc[f"threads_{oracle.get_threads()}"] = {"voxels_per_s": len(f.test_key) / dt, "seconds": dt}
    return orc


def cpu_baseline(S_h, Q_h, n_sample, n_sample_1t):
    """The FP64 oracle on the host cores: the surface is binned once (timed on its own), then
    the first queries of the workload are answered on all cores and, on a smaller sample, on
    one thread."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    t0 = time.perf_counter()
    surf = oracle.Surface(S_h, oracle.params())
    t_build = time.perf_counter() - t0
    q = Q_h[:n_sample]
    t0 = time.perf_counter()
    surf.query(q, want_var=False)
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    q1 = Q_h[:n_sample_1t]
    t0 = time.perf_counter()
    surf.query(q1, want_var=False)
    dt1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    return {"value": len(q) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"first {len(q)} of the 10M queries against the full 2M-point surface; surface binned "
                       f"once beforehand ({t_build:.2f} s, not included)"),
            "seconds": dt, "surface_build_s": t_build,
            "single_thread": {"value": len(q1) / dt1, "unit": UNIT, "cores": 1, "sample": f"first {len(q1)} queries",
                              "seconds": dt1}}


def error_vs_oracle(S_h, Q_h, m, n_sample):
    """The headline configuration's outputs (mixed precision, the benchmark's map, variance on)
    against the FP64 oracle on the CPU-baseline sample: max |d - d_ref| by distance bin,
    gradient angle, relative variance error, status agreement."""
    import oracle
    import torch
    q = Q_h[:n_sample]
    ref = oracle.Surface(S_h, oracle.params()).query(q, want_var=True)
    m.set_surface(torch.from_numpy(S_h).cuda())
    got = {k: v.cpu().numpy() for k, v in m.query(torch.from_numpy(q).cuda(), grad=True, var=True).items()}
    ok = (got["status"] == 0) & (ref["status"] == 0)
    d, rd = got["d"][ok], ref["d"][ok]
    g, rg = got["grad"][ok], ref["grad"][ok]
    dd = np.abs(d - rd)
    bins = {}
    for lo, hi in ((0.0, 0.1), (0.1, 0.5), (0.5, 2.0), (2.0, np.inf)):
        sel = (rd >= lo) & (rd < hi)
        if sel.any():
            bins[f"{lo}-{hi}"] = {"n": int(sel.sum()), "max_abs_dd_m": float(dd[sel].max())}
    big = (rd > 0.05) & (np.linalg.norm(rg, axis=1) > 1e-3)
    cosang = np.sum(g[big] * rg[big], 1) / (np.linalg.norm(g[big], axis=1) * np.linalg.norm(rg[big], axis=1))
    ang = np.degrees(np.arccos(np.clip(cosang, -1.0, 1.0)))
    fin = np.isfinite(ref["var"][ok]) & (ref["var"][ok] > 0)
    rv = np.abs(got["var"][ok][fin] - ref["var"][ok][fin]) / ref["var"][ok][fin]
    return {"precision": "mixed", "queries": int(len(q)), "status_equal": bool(np.array_equal(got["status"], ref["status"])),
            "max_abs_dd_m": float(dd.max()), "by_distance_m": bins,
            "grad_angle_deg": {"max": float(ang.max()), "p99.9": float(np.percentile(ang, 99.9))},
            "var_rel_err": {"max": float(rv.max()), "median": float(np.median(rv))}}


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
    t0 = time.perf_counter()
    surf = oracle.Surface(S_h, oracle.params())
    t_build = time.perf_counter() - t0
    times = []
    for i in range(args.warmup + args.steps):
        q = Q_h[i * n:(i + 1) * n]
        t0 = time.perf_counter()
        surf.query(q, want_var=False)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    value = n / float(np.mean(times))
    sample = (f"{n} queries per step against the full 2M-point surface, binned once beforehand "
              f"({t_build:.2f} s, not included)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded city scene)",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "n_surface": int(S_h.shape[0]), "n_queries": int(Q_h.shape[0]),
                       "precision": "fp64 oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-surface", type=int, default=2_000_000)
    ap.add_argument("--n-query", type=int, default=10_000_000)
    ap.add_argument("--cpu-sample", type=int, default=2000, help="queries of the all-core oracle baseline")
    ap.add_argument("--cpu-sample-1t", type=int, default=200, help="queries of the one-thread oracle baseline")
    ap.add_argument("--ref-sample", type=int, default=1000)
    ap.add_argument("--quick", action="store_true", help="skip the comparison lines")
    ap.add_argument("--n-sub", type=int, default=1_000_000, help="queries of the precision comparison subset")
    ap.add_argument("--n-per-instance", type=int, default=5_000, help="queries of the per-instance comparison")
    ap.add_argument("--room-frames", type=int, default=50)
    ap.add_argument("--frame-reps", type=int, default=5)
    ap.add_argument("--n-tune", type=int, default=2_000_000, help="queries the autotuner times")
    ap.add_argument("--prof-steps", type=int, default=2, help="steps of the instrumented (profile) pass")
    ap.add_argument("--sweep-inst", type=int, default=200_000)
    ap.add_argument("--sweep-per-instance", type=int, default=1000,
                    help="instances of the per-instance FP64 comparison on the sweep")
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

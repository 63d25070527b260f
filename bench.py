"""Benchmark of the PPE hot path on GB300.

One step = one complete PPE solve to relative residual 1e-8 of the 512x512
refined-box workload (refined box [0.4, 0.6]^2, geometric growth 1.05,
random-Fourier source with 1/|k|^2 amplitudes up to |k| = 32), inputs
resident in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

``--impl reference`` times the FP64 CPU oracle (Jacobi PCG on the assembled
CSR matrix) on the host cores for the same workload and metric.
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
sys.path.insert(0, ROOT)

from paper_2604_01800_gb300 import inputs as I  # noqa: E402
from paper_2604_01800_gb300 import shard  # noqa: E402

METRIC = "PPE solves/s at rel-res 1e-8 (512x512 refined-box grid, mixed FP32/FP64 PCG)"
WEIGHTS = os.path.join(ROOT, "paper_2604_01800_gb300", "weights", "hydea_mconv.ppenet")
# DRAM bytes of one launch of the solver kernel on the 512x512 workload (one
# whole mixed-precision solve), from an ncu capture of the current kernel
SOLVER_C2_DRAM_BYTES = 4.397312e6 + 0.122624e6
TOL = 1e-8
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--no-sweep", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    return p.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def cpu_oracle_baseline(w, max_seconds=30.0, min_solves=1):
    """Time the FP64 CPU oracle on the host (single thread) on whole solves."""
    import oracle
    oracle.build()
    times = []
    t_start = time.perf_counter()
    while len(times) < min_solves or (time.perf_counter() - t_start < max_seconds * 0.5 and len(times) < 3):
        t0 = time.perf_counter()
        x, info, st = oracle.solve(w.dx, w.dy, w.f, tol_rel=TOL)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > max_seconds:
            break
    return {"value": 1.0 / float(np.median(times)), "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(times)} full solve(s) of the {w.nx}x{w.ny} workload to rel-res 1e-8, "
                      f"FP64 CSR Jacobi PCG, one host thread", "iters": info["iters"]}


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    w = I.config2(0)
    import oracle
    oracle.build()
    # one full solve gives the iteration count of the workload; each step is
    # then a bounded sample (a quarter of the iterations, a few seconds on one
    # host thread), scaled to solves/s by the fraction of a solve it covers
    _, full, _ = oracle.solve(w.dx, w.dy, w.f, tol_rel=TOL)
    cap = max(1, full["iters"] // 4)
    for _ in range(args.warmup):
        oracle.solve(w.dx, w.dy, w.f, tol_rel=1e-30, maxit=cap)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x, info, st = oracle.solve(w.dx, w.dy, w.f, tol_rel=1e-30, maxit=cap)
    dt = time.perf_counter() - t0
    v = args.steps * (cap / full["iters"]) / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "tol_rel": TOL,
                                             "solver": "CPU FP64 Jacobi PCG (oracle)"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} x {cap} of the {full['iters']} iterations of a full "
                                       f"solve, one host thread, scaled to solves/s"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_native(args):
    import torch
    import torch.distributed as dist

    from paper_2604_01800_gb300 import api

    rank, world, local = _dist()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()

    w = I.config2(rank)              # weak scaling: each rank solves its own system
    grid = api.ppe_create_grid(w.dx, w.dy)
    rhs = torch.tensor(w.f, dtype=torch.float64, device=dev)
    x = torch.zeros_like(rhs)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    prec = api.PPE_PREC_MIXED

    def solve_once():
        x.zero_()
        return api.ppe_solve(grid, rhs, x, TOL, api.PPE_MODE_PCG, prec)

    for _ in range(args.warmup):
        info = solve_once()
    torch.cuda.synchronize()

    # ---- device-resident timing: CUDA events around each solve, L2 flushed between
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    launches = 0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            x.zero_()
            ev[k][0].record(stream)
            info = api.ppe_solve(grid, rhs, x, TOL, api.PPE_MODE_PCG, prec)
            ev[k][1].record(stream)
            infos.append(info)
            launches += info["launches"]
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    t_total = shard.max_over_ranks(sum(ms) / 1e3, dev)
    value = world * args.steps / t_total
    for info in infos:
        assert info["status"] == 0 and info["rel_res_true"] <= TOL, info

    # ---- end-to-end: pinned host source in, host solution out, through the public API
    h_rhs = torch.tensor(w.f, dtype=torch.float64).pin_memory()
    h_x = torch.empty_like(h_rhs).pin_memory()
    d_rhs = torch.empty_like(rhs)
    d_x = torch.empty_like(rhs)
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        d_rhs.copy_(h_rhs, non_blocking=True)
        d_x.zero_()
        api.ppe_solve(grid, d_rhs, d_x, TOL, api.PPE_MODE_PCG, prec)
        h_x.copy_(d_x, non_blocking=True)
        torch.cuda.synchronize()
    e2e_dt = time.perf_counter() - t0
    e2e = {"value": world * e2e_steps / e2e_dt if world == 1 else None, "unit": "solves/s",
           "h2d_bytes_per_step": int(h_rhs.numel() * 8), "d2h_bytes_per_step": int(h_x.numel() * 8)}
    if world > 1:
        e2e["value"] = world * e2e_steps / shard.max_over_ranks(e2e_dt, dev)

    # ---- roofline of the dominant kernel (the persistent solver kernel)
    peaks, peak_src = _peaks()
    it = float(np.mean([i["iters_pcg"] for i in infos]))
    ref = float(np.mean([i["refinements"] for i in infos]))
    n = w.nx * w.ny
    alg_bytes = n * (24.0 * it + 24.0 * ref)       # FP32 iterations + FP64 residual passes
    achieved = alg_bytes / (t_total / args.steps) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": SOLVER_C2_DRAM_BYTES,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch (one solve), "
                              "profiles/solver_kernel_tile_c2.md",
            "kernel": "solver_kernel<float>", "peak_source": f"hbm_gbs ({peak_src})",
            "note": "working set (~10 MB) is L2-resident: latency/barrier-bound, not HBM-bound"}

    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "tol_rel": TOL, "mode": "pcg",
                       "precision": "mixed FP32 inner / FP64 refinement", "l2": "flushed between steps",
                       "spacing_ratio": round(I.spacing_ratio(w.dx, w.dy), 2)},
            "iters_per_solve": it, "refinements_per_solve": ref,
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "clocks": clk.summary()}

    if not args.no_sweep and rank == 0:
        line["stencil_sweep"] = stencil_sweep(api, dev, peaks)
    if rank == 0:
        line["hybrid_vs_plain"] = hybrid_vs_plain(api, dev, flush)
    batch = batch_vs_sequential(api, dev, flush, peaks, rank, world)      # every rank: its share
    if rank == 0:
        line["batch_vs_sequential"] = batch
        line["sequence_c5"] = sequence_c5(api, dev, flush)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def hybrid_vs_plain(api, dev, flush, reps=5):
    """HyDEA (Jacobi PCG + DLSM with a trained network) against plain PCG on
    the 256x256 cylinder-refined grid with masked-divergence sources, all in
    mixed precision, to rel-res 1e-8 (median of `reps` sources each), with
    the network trained on random stretched grids."""
    import torch
    if not os.path.exists(WEIGHTS):
        return {"available": False, "reason": "no trained weights file"}
    nets = {"hybrid": api.net_load(WEIGHTS)}
    out = {"workload": "cyl256_mask (256x256, cylinder D=0.1, box-refined, growth 1.05)"}
    rows = {k: [] for k in ["pcg", *nets]}
    for i in range(reps):
        w = I.config3(i)
        g = api.ppe_create_grid(w.dx, w.dy, w.mask)
        rhs = torch.tensor(w.f, dtype=torch.float64, device=dev)
        for key in rows:
            net = nets.get(key)
            mode = api.PPE_MODE_PCG if net is None else api.PPE_MODE_HYBRID
            if net is not None:
                net.attach(g)
            x = torch.zeros_like(rhs)
            api.ppe_solve(g, rhs, x, TOL, mode, api.PPE_PREC_MIXED, net=net)     # warm (graph capture)
            flush.fill_(1.0)
            x.zero_()
            rows[key].append(api.ppe_solve(g, rhs, x, TOL, mode, api.PPE_PREC_MIXED, net=net))
        g.close()
    for key, infos in rows.items():
        ms = float(np.median([i["ms_total"] for i in infos]))
        out[key] = {"solves_per_s": 1e3 / ms, "ms_median": ms,
                    "iters_median": float(np.median([i["iters_pcg"] + i["iters_dlsm"] for i in infos])),
                    "dlsm_steps_median": float(np.median([i["iters_dlsm"] for i in infos])),
                    "fell_back": int(sum(i["fell_back"] for i in infos)),
                    "max_rel_res": float(max(i["rel_res_true"] for i in infos))}
    out["speedup"] = out["hybrid"]["solves_per_s"] / out["pcg"]["solves_per_s"]
    for net in nets.values():
        net.close()
    return out


def sequence_c5(api, dev, flush, steps=16):
    """The projection loop's use of the solver on the 2048x1024 wake-refined
    cylinder grid: one solve per time step to rel-res 1e-8, warm-started from
    the previous step's solution, plain mixed PCG and the hybrid each on its
    own chain.  The first `steps` of the 500-step sequence (sources built on
    the host before timing); solve times are device-timed."""
    import torch
    dx, dy, bodies = I.config5_grid()
    grid = api.ppe_create_grid(dx, dy)
    srcs = [I.config5_rhs(t, dx, dy, bodies) for t in range(steps)]
    arms = {"pcg": None}
    if os.path.exists(WEIGHTS):
        arms["hybrid"] = api.net_load(WEIGHTS)
    out = {"workload": f"cyl2048x1024 wake-refined (spacing ratio {I.spacing_ratio(dx, dy):.1f}), "
                       f"first {steps} of 500 steps, warm starts", "cells": int(dx.size * dy.size)}
    for key, net in arms.items():
        if net is not None:
            net.attach(grid)
        mode = api.PPE_MODE_PCG if net is None else api.PPE_MODE_HYBRID
        x = torch.zeros(dy.size, dx.size, dtype=torch.float64, device=dev)
        rhs = torch.empty_like(x)
        rhs.copy_(torch.from_numpy(srcs[0]))
        api.ppe_solve(grid, rhs, torch.zeros_like(x), TOL, mode, api.PPE_PREC_MIXED, net=net)   # warm-up
        infos = []
        for f in srcs:
            rhs.copy_(torch.from_numpy(f))
            flush.fill_(2.0)
            infos.append(api.ppe_solve(grid, rhs, x, TOL, mode, api.PPE_PREC_MIXED, net=net))
        ms = [i["ms_total"] for i in infos]
        out[key] = {"total_ms": float(sum(ms)), "ms_per_step": float(np.mean(ms)),
                    "iters_per_step": float(np.mean([i["iters_pcg"] + i["iters_dlsm"] for i in infos])),
                    "dlsm_steps": int(sum(i["iters_dlsm"] for i in infos)),
                    "fell_back": int(sum(i["fell_back"] for i in infos)),
                    "max_rel_res": float(max(i["rel_res_true"] for i in infos)),
                    "all_ok": bool(all(i["status"] == 0 for i in infos))}
        if net is not None:
            net.close()
    if "hybrid" in out:
        out["speedup"] = out["pcg"]["total_ms"] / out["hybrid"]["total_ms"]
    grid.close()
    return out


def batch_vs_sequential(api, dev, flush, peaks, rank=0, world=1, count=64):
    """64 independent systems (n ~ U{128..768}, random stretching, 0-3
    obstacles, masked-divergence sources) in one persistent launch against 64
    sequential ppe_solve calls; mixed precision, rel-res 1e-8.  With several
    ranks each solves its share (greedy balance on estimated cost) and the
    slowest rank's time counts."""
    import torch
    ws_all = I.config4(count)
    mine = shard.partition([shard.system_cost(w.nx, w.ny) for w in ws_all], world)[rank]
    ws = [ws_all[i] for i in mine]
    grids = [api.ppe_create_grid(w.dx, w.dy, w.mask) for w in ws]
    rhs = [torch.tensor(w.f, dtype=torch.float64, device=dev) for w in ws]
    xs = [torch.zeros_like(r) for r in rhs]
    cells = sum(w.nx * w.ny for w in ws)

    def batch():
        for x in xs:
            x.zero_()
        flush.fill_(2.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        infos, st = api.ppe_solve_batch(grids, rhs, xs, TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3, infos

    def sequential():
        for x in xs:
            x.zero_()
        flush.fill_(3.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        infos = [api.ppe_solve(g, r, x, TOL, api.PPE_MODE_PCG, api.PPE_PREC_MIXED) for g, r, x in zip(grids, rhs, xs)]
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3, infos

    batch()
    tb, ib = min((batch() for _ in range(2)), key=lambda t: t[0])
    ts, iseq = sequential()
    for g in grids:
        g.close()
    # algorithmic bytes of the batch: 24 B per cell per FP32 iteration, 24 B per FP64 residual pass
    mine_rep = {"ok": all(i["status"] == 0 and i["rel_res_true"] <= TOL for i in ib), "cells": cells,
                "iters": [i["iters_pcg"] for i in ib],
                "alg": sum(w.nx * w.ny * 24.0 * (i["iters_pcg"] + i["refinements"]) for w, i in zip(ws, ib))}
    tb, ts = shard.max_over_ranks(tb, dev), shard.max_over_ranks(ts, dev)
    reps = shard.gather_to_rank0(mine_rep)
    if rank != 0:
        return None
    iters = [k for r in reps for k in r["iters"]]
    alg = sum(r["alg"] for r in reps)
    return {"systems": count, "ranks": world, "cells": sum(r["cells"] for r in reps),
            "all_converged": all(r["ok"] for r in reps),
            "batch_seconds": tb, "batch_systems_per_s": count / tb,
            "sequential_seconds": ts, "sequential_systems_per_s": count / ts, "speedup": ts / tb,
            "max_iters": max(iters), "mean_iters": float(np.mean(iters)),
            "effective_gbs": alg / tb / 1e9, "frac_of_hbm": alg / tb / 1e9 / peaks["hbm_gbs"] / world}


def stencil_sweep(api, dev, peaks, sizes=(4096, 8192, 16384), short=20, long=120):
    """Per-iteration cost of the FP32 PCG iteration pass on grids far above L2:
    two solves capped at `short` and `long` iterations (no residual
    replacement in between), timed with CUDA events; the difference divided by
    the extra iterations is the cost of one iteration pass over the grid."""
    import torch
    out = []
    for n in sizes:
        dx = I.box_spacing(n, 0.4, 0.6, 1.01)
        g = api.ppe_create_grid(dx, dx)
        xc = np.cumsum(dx) - 0.5 * dx
        gx = np.cos(np.pi * xc) + 0.3 * np.cos(3 * np.pi * xc)
        gx -= np.dot(dx, gx) / dx.sum()         # volume-weighted zero mean: a compatible source
        rhs = torch.outer(torch.tensor(gx, device=dev), torch.tensor(gx, device=dev)).contiguous()
        for iter_pass in (1, 2):
            out.append(_sweep_one(api, g, rhs, n, iter_pass, short, long, peaks))
        g.close()
        del rhs
    return {"alg_bytes_per_cell_iter": 24, "method": f"(t[{long} its] - t[{short} its]) / extra iterations",
            "grids": out}


def _sweep_one(api, g, rhs, n, iter_pass, short, long, peaks):
    import torch
    x = torch.zeros_like(rhs)
    t, info = {}, {}
    for cap in (short, long):
        api.ppe_set_options(g, max_iters=cap, inner_rtol=1e-12, iter_pass=iter_pass)
        api.ppe_solve(g, rhs, x, 1e-14, api.PPE_MODE_PCG, api.PPE_PREC_MIXED, raise_on_error=False)
        times = []
        for _ in range(3):
            x.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            info[cap] = api.ppe_solve(g, rhs, x, 1e-14, api.PPE_MODE_PCG, api.PPE_PREC_MIXED, raise_on_error=False)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b) / 1e3)
        t[cap] = min(times)
    d_it = info[long]["iters_pcg"] - info[short]["iters_pcg"]
    same_ref = info[long]["refinements"] == info[short]["refinements"]
    t_it = (t[long] - t[short]) / max(d_it, 1)
    gbs = 24.0 * n * n / t_it / 1e9
    return {"grid": f"{n}x{n}", "iter_pass": ["", "tile", "stream"][iter_pass], "us_per_iter": 1e6 * t_it,
            "achieved_gbs": gbs, "frac_of_hbm": gbs / peaks["hbm_gbs"], "extra_iters": d_it,
            "same_refinements": same_ref}


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()

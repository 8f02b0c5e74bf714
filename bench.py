#!/usr/bin/env python
"""Throughput of the compressed-sensing PAT operators: A + A^T pairs per second.

Workload (default `c2`): 64x128x128 grid (z, y, x), dx = 100 um, c = 1500 m/s, CFL 0.3 (dt = 20 ns),
T = 400 recorded steps, 10-voxel PML, random single-point sampling of 2048 of the 16384 detection
plane points, a 20-tube synthetic vessel phantom.  One step = one forward A (p0 -> f = C A p0)
plus one adjoint (f -> A^T C^T f) on each of `--batch` independent volumes, inputs resident on the
GPU.  Between steps a 256 MiB buffer is written (inside the timed region) so that no step starts
with the previous step's data in the 129 MB L2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--workload c2]
    python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores, same metric

Multi-GPU: replicas only (torchrun, one rank per GPU, independent volumes, no collective on the
data path); value = pairs processed by all ranks / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "A+A^T pairs/s (64x128x128, 400 steps)"

# (kernel source hash, workload, batch) -> DRAM bytes (read + write) of one time step, from ncu
STEP_TRAFFIC = {("7a22aba1b07a", "c2", 1): 53.54e6}
UNIT = "pairs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--solve", action="store_true",
                    help="also time one TV-Bregman reconstruction of the workload (reported, not the metric)")
    ap.add_argument("--warm", action="store_true",
                    help="also train the learned warm start and time warm vs plain solves to 2 %% error")
    ap.add_argument("--warm-train", type=int, default=64)
    ap.add_argument("--warm-test", type=int, default=4)
    ap.add_argument("--warm-epochs", type=int, default=20)
    return ap.parse_args()


def workload_config(w, batch):
    g, s = w.grid, w.sampling
    kinds = {0: "full plane", 1: "rSP", 2: "sHd 0/1", 3: "sHd +-1"}
    return {
        "workload": (f"{w.name}: {g.nz}x{g.ny}x{g.nx} (z,y,x), dx {g.dx * 1e6:g} um, c {g.c:g} m/s, "
                     f"CFL {g.cfl:g} (dt {g.dt * 1e9:g} ns), T {g.T}, {g.pml_size}-pt PML, "
                     f"{kinds[s.kind]} {s.m}/{g.m_plane}, {w.phantom} phantom"),
        "batch": batch,
        "step": "one forward A and one adjoint A^T per volume",
        "l2_flush": "256 MiB buffer written between steps, inside the timed region",
    }


# ------------------------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        sm_sorted = sorted(sm)
        med = sm_sorted[len(sm_sorted) // 2] if sm_sorted else None
        return {"sm_mhz": med, "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ------------------------------------------------------------------------------------ CPU oracle

def oracle_pairs_per_s(w, n_steps_sample):
    """Time the FP64 oracle's A + A^T on the full grid with n_steps_sample recorded steps and scale to
    the full T by the step count.  Returns (pairs/s, seconds, threads)."""
    import numpy as np

    import oracle
    from paper_1605_00133_gb300 import presets
    ws = presets.shrink(w, n_steps_sample)
    g, s = ws.grid, ws.sampling
    p0 = w.p0()
    y = np.random.default_rng(0).standard_normal((g.T, s.m))
    t0 = time.perf_counter()
    oracle.forward(g, s, p0)
    oracle.adjoint(g, s, y)
    t = time.perf_counter() - t0
    scale = (w.grid.T - 1) / (n_steps_sample - 1)
    return 1.0 / (t * scale), t, oracle.num_threads()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_1605_00133_gb300 import presets
    oracle.build()
    w = presets.workload(args.workload)
    Ts = 4
    for _ in range(args.warmup):
        oracle_pairs_per_s(w, Ts)
    tot = 0.0
    for _ in range(args.steps):
        _, t, threads = oracle_pairs_per_s(w, Ts)
        tot += t
    scale = (w.grid.T - 1) / (Ts - 1)
    sec_per_pair = tot / args.steps * scale
    value = 1.0 / sec_per_pair
    sample = (f"each step: oracle A + A^T on the full {w.grid.nz}x{w.grid.ny}x{w.grid.nx} grid with "
              f"T = {Ts} ({Ts - 1} time steps each way), scaled by {scale:.1f} to T = {w.grid.T}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec_per_pair * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------ GPU arm

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    __graft_entry__.build()

    from paper_1605_00133_gb300 import presets, replicas
    from paper_1605_00133_gb300.operators import PatOperator

    w = presets.workload(args.workload)
    B = args.batch
    g = w.grid
    gb = presets.Grid(g.nz, g.ny, g.nx, dx=g.dx, c=g.c, rho0=g.rho0, cfl=g.cfl, T=g.T,
                      pml_size=g.pml_size, pml_alpha=g.pml_alpha, sensor_z=g.sensor_z, batch=B)
    op = PatOperator(gb, w.sampling)
    p0_np = np.stack([w.p0(seed_offset=o) for o in replicas.volume_seeds(rank, B)]).astype(np.float32)
    p0 = torch.tensor(p0_np, device=dev)
    f = torch.empty(op.data_shape, device=dev)
    p = torch.empty(op.image_shape, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    def step():
        op.forward_into(p0, f)
        op.adjoint_into(f, p)
        flush.fill_(1.0)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return replicas.max_over_ranks(x, dist, dev)

    for _ in range(args.warmup):
        step()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    barrier()
    ms = max_over_ranks(ms)
    pairs = B * world * args.steps
    value = replicas.whole_job_rate(B * args.steps, world, ms / 1e3)

    # per-kernel breakdown: the same K steps again with every launch bracketed by CUDA events on the
    # launching stream (torch's current stream, which the library uses)
    op.profile(True)
    for _ in range(args.steps):
        step()
    prof = op.profile_read()
    op.profile(False)
    total_prof = sum(v[0] for v in prof.values())
    launches_per_step = sum(v[1] for v in prof.values()) / args.steps
    kernels = {k: {"ms_total": v[0], "launches": v[1], "avg_us": 1e3 * v[0] / v[1],
                   "share": v[0] / total_prof} for k, v in prof.items()}
    dominant = max(kernels, key=lambda k: kernels[k]["ms_total"])

    # roofline: the time step is the unit of work (48 bytes per voxel per step: six FP32 state fields
    # read and written once); one step = 3 line-pass launches (x, y, z) on one stream
    import json as _json
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak, peak_src = 6800.0, "fallback 6.8 TB/s"
    if os.path.exists(peaks_path):
        pk = _json.load(open(peaks_path))
        peak, peak_src = float(pk["hbm_gbs"]), "measured hbm_gbs"
    steps_per_pair = 2 * (g.T - 1)
    step_s = (ms / 1e3) / (args.steps * steps_per_pair)
    bytes_per_step = 48.0 * g.n * B
    achieved = bytes_per_step / step_s / 1e9
    # DRAM bytes of one forward time step from the committed ncu capture, valid only for the kernel
    # sources it was taken on (profiles/pat_line_pass_c2.md)
    traffic = STEP_TRAFFIC.get((_source_hash(), w.name, B))
    roofline = {"bound": "hbm", "kernel": "time step (line passes x, y, z of A, and of A^T)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": peak_src,
                "algorithmic_bytes_per_unit": "48 B per voxel per time step",
                "dominant_kernel": dominant, "dominant_share": kernels[dominant]["share"],
                "dominant_avg_us": kernels[dominant]["avg_us"]}

    # second roofline: the conventional scheme's algorithmic flops, ten real 3D FFTs
    # (2.5 N log2 N each) plus ~60 N pointwise per time step, against the FP32 FMA peak of the CUDA
    # cores from unit counts and clock (152 SMs x 128 lanes x 2 flops x max SM clock)
    import math
    flops_per_step = 10 * 2.5 * g.n * math.log2(g.n) + 60.0 * g.n
    sm_mhz = clk.get("sm_max_mhz") or 2070.0
    alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    alu_achieved = flops_per_step * B / step_s / 1e12
    roofline_alu = {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": alu_achieved / alu_peak,
                    "algorithmic_flops_per_unit": "10 x 2.5 N log2 N + 60 N per time step",
                    "peak_source": "152 SMs x 128 FP32 lanes x 2 x max SM clock"}

    # end to end through the public API: pinned host p0 -> device, A, A^T, device -> pinned host
    e2e = None
    if not args.no_e2e:
        p0_h = torch.tensor(p0_np).pin_memory()
        p_h = torch.empty(op.image_shape, dtype=torch.float32).pin_memory()
        p0_d = torch.empty_like(p0)

        def step_e2e():
            p0_d.copy_(p0_h, non_blocking=True)
            op.forward_into(p0_d, f)
            op.adjoint_into(f, p)
            p_h.copy_(p, non_blocking=True)
            flush.fill_(1.0)

        for _ in range(max(1, args.warmup)):
            step_e2e()
        barrier()
        e0.record()
        for _ in range(args.steps):
            step_e2e()
        e1.record()
        torch.cuda.synchronize()
        ms_e2e = max_over_ranks(e0.elapsed_time(e1))
        e2e = {"value": pairs / (ms_e2e / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(p0_h.numel() * 4), "d2h_bytes_per_step": int(p_h.numel() * 4)}

    solve = None
    if args.solve and B == 1:
        # one TV+Br reconstruction (outer x inner FISTA steps, each one A + A^T pair plus restarts),
        # then the plain solve's time to 2 % relative error against its own final image: the solves
        # with k = 1, 2, ... Bregman steps (deterministic, so solve k ends at the k-th iterate of the
        # full solve), each timed from scratch
        from paper_1605_00133_gb300.presets import workload as _wl
        wl = _wl(args.workload)
        fnoisy = f + 0.01 * float(f.abs().max()) * torch.randn(f.shape, device=dev,
                                                                generator=torch.Generator(device=dev).manual_seed(5))
        lam = 2e-4

        def timed_solve(outer):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pr, rp = op.bregman_solve(fnoisy, lam, outer=outer, inner=wl.inner, prox_iters=50, power_iters=20)
            torch.cuda.synchronize()
            return pr, rp, time.perf_counter() - t0

        prec, rep, secs = timed_solve(wl.bregman_outer)
        traj = []
        for k in range(1, wl.bregman_outer):
            pk, _, tk = timed_solve(k)
            traj.append({"bregman_steps": k, "seconds": tk,
                         "rel_err_vs_final": float((pk - prec).norm() / prec.norm())})
        traj.append({"bregman_steps": wl.bregman_outer, "seconds": secs, "rel_err_vs_final": 0.0})
        t2 = next(t["seconds"] for t in traj if t["rel_err_vs_final"] <= 0.02)
        solve = {"seconds": secs, "reconstructions_per_min": 60.0 / secs, "outer": wl.bregman_outer,
                 "inner": wl.inner, "prox_iters": 50, "lambda": lam, "power_iters": 20,
                 "fista_iterations": rep["inner_total"], "restarts": rep["restarts"],
                 "residuals": rep["residuals"], "rel_err_vs_phantom": float((prec - p0).norm() / p0.norm()),
                 "plain_seconds_to_2pct": t2, "trajectory": traj,
                 "warm_start": "plain cold-start solve; --warm trains the learned U-Net warm start and "
                               "times warm against plain (the line's warm_start object)"}

    warm = None
    if args.warm and B == 1:
        warm = warm_start_experiment(args, op, g, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        Ts = 100
        v, t, threads = oracle_pairs_per_s(w, Ts)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": (f"one oracle A + A^T on the full {g.nz}x{g.ny}x{g.nx} grid with T = {Ts} "
                          f"({Ts - 1} time steps each way, {t:.1f} s), scaled to T = {g.T}")}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(w, B), "clocks": clk, "e2e": e2e,
                "gpu_launches": int(round(launches_per_step * args.steps)),
                "roofline": roofline, "roofline_alu": roofline_alu, "kernels": kernels, "cpu_baseline": cpu}
        if solve is not None:
            line["solve"] = solve
        if warm is not None:
            line["warm_start"] = warm
        print(json.dumps(line), flush=True)
    op.close()
    if dist:
        dist.destroy_process_group()
    return 0


def warm_start_experiment(args, op, g, dev):
    """Train the U-Net warm start on seeded phantoms of the workload and compare warm vs plain solves
    on held-out phantoms (time to 2 % relative error against the plain solve's final image)."""
    import numpy as np
    import torch

    from paper_1605_00133_gb300 import presets, unet, warmstart
    wl = presets.workload(args.workload)
    lam = 2e-4
    # the step size 1/L (power iteration) once per grid, shared by every solve below
    _, rep = op.bregman_solve(torch.zeros(op.data_shape, device=dev), lam, outer=1, inner=1, prox_iters=1,
                              power_iters=20)
    L = rep["L"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    train_pairs = warmstart.make_pairs(op, wl, args.warm_train, 1000, lam, wl.bregman_outer, wl.inner, L)
    test_pairs = warmstart.make_pairs(op, wl, args.warm_test, 5000, lam, wl.bregman_outer, wl.inner, L)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = unet.WarmStartUNet(g.nz, g.ny, g.nx, seed=0)
    net.s_in = warmstart.input_scale(train_pairs)
    t0 = time.perf_counter()
    hist = warmstart.train(net, train_pairs, args.warm_epochs, lr=1e-3, seed=0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    steps = args.warm_epochs * len(train_pairs)
    inners = [10, 20, 30, 40, wl.inner]
    ev = warmstart.evaluate(op, net, test_pairs, lam, wl.bregman_outer, inners, L)
    t_plain = [e["plain_seconds_to_tol"] for e in ev]
    t_warm = [e["warm_seconds_to_tol"] for e in ev]

    def med(v):
        v = [x for x in v if x is not None]
        return float(np.median(v)) if v else None
    return {"train_pairs": len(train_pairs), "test_pairs": len(test_pairs), "epochs": args.warm_epochs,
            "train_steps": steps, "train_seconds": t_train, "train_ms_per_step": 1e3 * t_train / steps,
            "data_seconds": t_data, "loss_per_epoch": hist, "L": L, "lambda": lam,
            "schedule": {"outer": wl.bregman_outer, "inner": inners, "tol": 0.02},
            "network_rel_err": [e["network_rel_err"] for e in ev],
            "inference_seconds": [e["inference_seconds"] for e in ev],
            "plain_seconds_to_2pct": t_plain, "warm_seconds_to_2pct": t_warm,
            "median_plain_seconds_to_2pct": med(t_plain), "median_warm_seconds_to_2pct": med(t_warm),
            "trajectories": [{"plain": e["plain"], "warm": e["warm"]} for e in ev]}


# sources that do not take part in A or A^T (solver, learned warm start): excluded from the hash
_NOT_OPERATOR = ("pat_solver.cu", "pat_unet.cu")


_C_TOKENS = re.compile(r'"(?:\\.|[^"\\])*"|//[^\n]*|/\*.*?\*/', re.S)


def _code_only(text: str) -> str:
    """C/C++/CUDA source with comments removed and whitespace collapsed (string literals kept)."""
    text = _C_TOKENS.sub(lambda m: m.group(0) if m.group(0).startswith('"') else " ", text)
    return " ".join(text.split())


def _source_hash():
    """sha1 of the operator's kernel sources (csrc/*.cu, *.cuh, *.h except _NOT_OPERATOR) with
    comments and whitespace left out, 12 digits: edits to comments keep the ncu figures valid"""
    import hashlib
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_1605_00133_gb300", "csrc")
    for n in sorted(os.listdir(d)):
        if n.endswith((".cu", ".cuh", ".h")) and n not in _NOT_OPERATOR:
            h.update(n.encode())
            h.update(_code_only(open(os.path.join(d, n), encoding="utf-8").read()).encode())
    return h.hexdigest()[:12]


if __name__ == "__main__":
    sys.exit(main())

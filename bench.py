#!/usr/bin/env python
"""Throughput of the compressed-sensing PAT operators: A + A^T pairs per second.

Workload (default `c2`): 64x128x128 grid (z, y, x), dx = 100 um, c = 1500 m/s, CFL 0.3 (dt = 20 ns),
T = 400 recorded steps, 10-voxel PML, random single-point sampling of 2048 of the 16384 detection
plane points, a 20-tube synthetic vessel phantom.  One step = one forward A (p0 -> f = C A p0)
plus one adjoint (f -> A^T C^T f) on each of `--batch` independent volumes, inputs resident on the
GPU.  Between steps a 256 MiB buffer is written (inside the timed region) so that no step starts
with the previous step's data in the 129 MB L2.

The metric's second half (the `solve` object, on by default at batch 1): one TV-Bregman
reconstruction with the workload's schedule (seconds, reconstructions per minute) and the plain
solve's time to 2 % relative error against a converged reconstruction.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--workload c2] [--no-solve]
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

# (kernel source hash, workload, batch) -> DRAM bytes (read + write) of one forward time step (x, y and
# z passes), from ncu with the L2 as the run leaves it (--cache-control none)
STEP_TRAFFIC = {("00f5b3bcbe10", "c2", 1): 4.84e6, ("00f5b3bcbe10", "c4", 1): 672.3e6}
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
    ap.add_argument("--no-batch-scan", action="store_true",
                    help="skip the timing of 2 and 4 volumes per call (the `batch_scan` object)")
    ap.add_argument("--no-solve", action="store_true",
                    help="skip the TV-Bregman reconstruction timing (the `solve` object)")
    ap.add_argument("--unet", action="store_true",
                    help="also time the learned warm start's U-Net (inference and one training step) at the "
                         "workload's grid: its tensor-core convolutions against the BF16 roofline")
    ap.add_argument("--unet-only", action="store_true",
                    help="only the U-Net timing (no operator timing, solve or CPU baseline)")
    ap.add_argument("--prox-only", action="store_true",
                    help="only the TV prox's timing at the workload's grid (50 primal-dual iterations on the "
                         "back-projection of the workload's data; the `solve.prox` object alone)")
    ap.add_argument("--warm", action="store_true",
                    help="also train the learned warm start and time warm vs plain solves to 2 %% error")
    ap.add_argument("--warm-train", type=int, default=256)
    ap.add_argument("--warm-test", type=int, default=3)
    ap.add_argument("--warm-epochs", type=int, default=20)
    ap.add_argument("--warm-target-inner", type=int, default=100,
                    help="FISTA iterations per Bregman step of the training targets")
    ap.add_argument("--warm-ref-inner", type=int, default=600,
                    help="FISTA iterations per Bregman step of the converged reference")
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
    Ts = 24  # 23 time steps each way: the per-call set-up is under 5 % of a sample
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
                             "sample": sample, "cpu_model": cpu_model(), "nproc": os.cpu_count()},
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
    if args.unet_only:
        if rank == 0:
            print(json.dumps({"metric": "U-Net training steps/s", "unet": unet_experiment(args, g, dev)}), flush=True)
        return 0
    gb = presets.Grid(g.nz, g.ny, g.nx, dx=g.dx, c=g.c, rho0=g.rho0, cfl=g.cfl, T=g.T,
                      pml_size=g.pml_size, pml_alpha=g.pml_alpha, sensor_z=g.sensor_z, batch=B)
    op = PatOperator(gb, w.sampling)
    p0_np = np.stack([w.p0(seed_offset=o) for o in replicas.volume_seeds(rank, B)]).astype(np.float32)
    p0 = torch.tensor(p0_np, device=dev)
    f = torch.empty(op.data_shape, device=dev)
    p = torch.empty(op.image_shape, device=dev)
    if args.prox_only:
        op.forward_into(p0, f)
        op.adjoint_into(f, p)
        alpha = 1e-3 * float(p.abs().max())
        res = prox_timing(op, p, alpha, 50)
        op.device_status(dev)
        if rank == 0:
            print(json.dumps({"metric": "TV prox us per iteration", "config": {"workload": w.name},
                              "alpha": alpha, "prox": res}), flush=True)
        return 0
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
    op.device_status(dev)  # raises if a bounded device-side wait gave up (results invalid)
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
    op.device_status(dev)
    total_prof = sum(v[0] for v in prof.values())
    launches_per_step = sum(v[1] for v in prof.values()) / args.steps
    kernels = {k: {"ms_total": v[0], "launches": v[1], "avg_us": 1e3 * v[0] / v[1],
                   "share": v[0] / total_prof} for k, v in prof.items()}
    kernels_note = ("serialised run: the same steps again with every launch bracketed by CUDA events, "
                    "which removes the overlap of successive launches; per-launch times and shares of "
                    "that run, not a decomposition of ms_per_step")
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
    # sources it was taken on
    traffic = STEP_TRAFFIC.get((_source_hash(), w.name, B))
    roofline = {"bound": "hbm", "kernel": "time step (line passes x, y, z of A, and of A^T)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_unit": "DRAM bytes (read + write) of one time step, ncu, warm L2",
                "peak_source": peak_src,
                "algorithmic_bytes_per_unit": "48 B per voxel per time step",
                "dominant_kernel": dominant, "dominant_share": kernels[dominant]["share"],
                "dominant_avg_us": kernels[dominant]["avg_us"]}

    # second roofline: the FP32 arithmetic this method executes per time step, against the FP32 FMA
    # peak of the CUDA cores from unit counts and clock (152 SMs x 128 lanes x 2 flops x max SM clock)
    flops_per_step = method_flops_per_step(g)
    sm_mhz = clk.get("sm_max_mhz") or 2070.0
    alu_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
    alu_achieved = flops_per_step * B / step_s / 1e12
    roofline_alu = {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": alu_achieved / alu_peak, "flops_per_unit": flops_per_step,
                    "algorithmic_flops_per_unit": ("per time step, per axis i: 4 complex line transforms "
                                                   "(5 L_i log2 L_i flops each) on the axis's lines, and "
                                                   "38 flops per line point (three k-space factors, two "
                                                   "state updates, the accumulation)"),
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
        op.device_status(dev)
        ms_e2e = max_over_ranks(e0.elapsed_time(e1))
        e2e = {"value": pairs / (ms_e2e / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(p0_h.numel() * 4), "d2h_bytes_per_step": int(p_h.numel() * 4)}

    solve = None
    if not args.no_solve and B == 1:
        solve = solve_experiment(args, op, f, p0, dev)
        op.device_status(dev)

    unet_line = unet_experiment(args, g, dev) if args.unet else None

    # the same step with 2 and 4 independent volumes per call (volume-pairs/s): B = 1 is the
    # line's value; these show what batching gains
    batch_scan = None
    if B == 1 and world == 1 and not args.no_batch_scan:
        batch_scan = {"1": value}
        for nb in (2, 4):
            gbn = presets.Grid(g.nz, g.ny, g.nx, dx=g.dx, c=g.c, rho0=g.rho0, cfl=g.cfl, T=g.T,
                               pml_size=g.pml_size, pml_alpha=g.pml_alpha, sensor_z=g.sensor_z, batch=nb)
            opn = PatOperator(gbn, w.sampling)
            p0n = torch.tensor(np.stack([w.p0(seed_offset=o) for o in range(nb)]).astype(np.float32), device=dev)
            fn = torch.empty(opn.data_shape, device=dev)
            pn = torch.empty(opn.image_shape, device=dev)

            def step_n():
                opn.forward_into(p0n, fn)
                opn.adjoint_into(fn, pn)
                flush.fill_(1.0)
            for _ in range(args.warmup):
                step_n()
            torch.cuda.synchronize()
            e0.record()
            for _ in range(args.steps):
                step_n()
            e1.record()
            torch.cuda.synchronize()
            opn.device_status(dev)
            batch_scan[str(nb)] = nb * args.steps / (e0.elapsed_time(e1) / 1e3)
            opn.close()
            del p0n, fn, pn

    warm = None
    if args.warm and B == 1:
        warm = warm_start_experiment(args, op, g, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(w, B), "clocks": clk, "e2e": e2e,
                "gpu_launches": int(round(launches_per_step * args.steps)),
                "roofline": roofline, "roofline_alu": roofline_alu, "kernels": kernels,
                "kernels_note": kernels_note, "cpu_baseline": cpu}
        if solve is not None:
            line["solve"] = solve
        if warm is not None:
            line["warm_start"] = warm
        if unet_line is not None:
            line["unet"] = unet_line
        if batch_scan is not None:
            line["batch_scan"] = {"unit": "volume-pairs/s", "volumes_per_call": batch_scan}
        print(json.dumps(line), flush=True)
    op.close()
    if dist:
        dist.destroy_process_group()
    return 0


def method_flops_per_step(g):
    """FP32 flops of one time step of the mixed-representation scheme: for each axis i, the lines of
    that axis (the half spectrum's columns along it) take four complex length-L_i transforms
    (5 L log2 L flops each, the radix-2 count) and 38 flops per line point (three complex k-space
    factors at 8, two state updates at 6, the spectrum accumulation at 2)."""
    import math
    nzh, nxh = g.nz // 2 + 1, g.nx // 2 + 1
    total = 0.0
    for L, n_lines in ((g.nz, nxh * g.ny), (g.ny, g.nz * nxh), (g.nx, nzh * g.ny)):
        total += n_lines * (4 * 5 * L * math.log2(L) + 38 * L)
    return total


def solve_experiment(args, op, f_clean, p0, dev):
    """The metric's second half on the workload (noisy data: f + 1 % Gaussian noise).

    * One TV-Bregman reconstruction with the workload's schedule (outer x inner FISTA steps, each one
      A + A^T pair plus restarts; the step size from 20 power iterations inside the timed call):
      seconds per reconstruction and reconstructions per minute.
    * The plain solve's time to 2 % relative error against p_ref, a converged reconstruction (the
      same solver, Bregman steps and prox iterations, 300 inner FISTA iterations per step, computed
      once and not timed): solves with an increasing number of inner iterations per Bregman step,
      each timed from scratch with the step size fixed, until one lands within 2 % of p_ref."""
    import torch

    from paper_1605_00133_gb300 import presets
    wl = presets.workload(args.workload)
    gen = torch.Generator(device=dev).manual_seed(5)
    f = f_clean + 0.01 * float(f_clean.abs().max()) * torch.randn(f_clean.shape, device=dev, generator=gen)
    lam, prox = 2e-4, 50

    def timed(inner, L=0.0, prox_iters=prox):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pr, rp = op.bregman_solve(f, lam, outer=wl.bregman_outer, inner=inner, prox_iters=prox_iters, L=L,
                                  power_iters=20)
        torch.cuda.synchronize()
        return pr, rp, time.perf_counter() - t0

    prec, rep, secs = timed(wl.inner)
    L = rep["L"]
    p_ref, rref, t_ref = timed(300, L)
    nref = float(p_ref.norm())
    ladder = []
    for inner in (10, 20, 50, 100, 150, 200):
        pk, rk, tk = timed(inner, L)
        ladder.append({"inner": inner, "seconds": tk, "fista_iterations": rk["inner_total"],
                       "rel_err_vs_ref": float((pk - p_ref).norm()) / nref})
        if ladder[-1]["rel_err_vs_ref"] <= 0.02:
            break
    t2 = next((e["seconds"] for e in ladder if e["rel_err_vs_ref"] <= 0.02), None)
    prox_rate = prox_timing(op, prec, lam * 1.8 / L, prox)
    seconds_to = {f"{tol:g}": next((e["seconds"] for e in ladder if e["rel_err_vs_ref"] <= tol), None)
                  for tol in (0.10, 0.05, 0.02)}
    return {"seconds": secs, "reconstructions_per_min": 60.0 / secs, "outer": wl.bregman_outer,
            "inner": wl.inner, "prox_iters": prox, "lambda": lam, "power_iters": 20, "L": L,
            "fista_iterations": rep["inner_total"], "restarts": rep["restarts"],
            "residuals": rep["residuals"], "rel_err_vs_phantom": float((prec - p0).norm() / p0.norm()),
            "rel_err_vs_ref": float((prec - p_ref).norm()) / nref,
            "reference": {"inner": 300, "prox_iters": prox, "fista_iterations": rref["inner_total"],
                          "seconds": t_ref},
            "plain_seconds_to_2pct": t2, "plain_seconds_to": seconds_to, "ladder": ladder,
            "prox": prox_rate,
            "warm_start": "plain cold-start solve; bench.py --warm trains the learned U-Net warm start and "
                          "times warm against plain against a 5 x 600 reference (the line's warm_start "
                          "object; about 55 GPU-minutes with the default 256 training phantoms)"}


def prox_timing(op, x, alpha, iters, reps=5):
    """The TV prox alone at the solver's alpha = eta lam: CUDA events around `reps` calls of `iters`
    fused primal-dual iterations (one launch each; a call's initial clamp and dual reset included).
    Algorithmic bytes per voxel and iteration: qbar, the three dual components, q and the input
    read, the dual, q and qbar written, 11 x 4 B = 44 B."""
    import json as _json

    import torch
    out = torch.empty_like(x)
    op.tv_prox(x, alpha, iters, out=out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        op.tv_prox(x, alpha, iters, out=out)
    e1.record()
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / (reps * iters)
    voxels = x.numel()
    gbs = 44.0 * voxels / (us * 1e-6) / 1e9
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak = float(_json.load(open(peaks_path))["hbm_gbs"]) if os.path.exists(peaks_path) else 6800.0
    fields = 10 * 4 * voxels  # qbar and the dual (3) in a read and a write buffer each, q, the input
    where = ("stay in the 129 MB L2 at this size, so the fraction is of the HBM copy bandwidth, not DRAM "
             "traffic") if fields < 100e6 else "exceed the L2 at this size"
    return {"iters": iters, "us_per_iter": us, "voxels": voxels, "algorithmic_bytes_per_voxel": 44,
            "achieved_gbs": gbs, "frac_of_hbm": gbs / peak,
            "note": f"one launch per iteration; the prox's fields (10 image-sized FP32 arrays, "
                    f"{fields / 1e6:.0f} MB) {where}"}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(w):
    """The FP64 oracle as it stands, on the host cores: the metric on a bounded sample of the workload
    (all cores), plus the timings of the survey's CPU plan: one pair of the 32^3 workload on all
    cores and on one, a 1-core sample of the workload, and a full oracle TV-Bregman solve of the
    32^3 workload (5 x 20 FISTA iterations), all timed, not extrapolated, except where marked."""
    import numpy as np

    import oracle
    from oracle import solver
    from paper_1605_00133_gb300 import presets, synth
    g = w.grid
    Ts = 100
    v, t, threads = oracle_pairs_per_s(w, Ts)
    out = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": (f"one oracle A + A^T on the full {g.nz}x{g.ny}x{g.nx} grid with T = {Ts} "
                      f"({Ts - 1} time steps each way, {t:.1f} s), scaled to T = {g.T}"),
           "cpu_model": cpu_model(), "nproc": os.cpu_count()}
    Ts1 = 8
    oracle.set_threads(1)
    v1, t1, _ = oracle_pairs_per_s(w, Ts1)
    out["one_core"] = {"value": v1, "unit": UNIT, "cores": 1,
                       "sample": f"T = {Ts1} ({t1:.1f} s), scaled to T = {g.T} (extrapolated)"}
    c1 = presets.workload("c1")
    gc, sc = c1.grid, c1.sampling
    p0 = c1.p0()
    y = np.random.default_rng(0).standard_normal((gc.T, sc.m))
    pair = {}
    for n in (1, threads):
        oracle.set_threads(n)
        t0 = time.perf_counter()
        oracle.forward(gc, sc, p0)
        oracle.adjoint(gc, sc, y)
        pair[n] = time.perf_counter() - t0
    oracle.set_threads(threads)
    out["c1_pair_seconds"] = {"one_core": pair[1], "all_cores": pair[threads],
                              "workload": "c1: 32^3, T 64, rSP 256/1024"}
    f = synth.add_relative_noise(oracle.forward(gc, sc, p0), 0.01, 4)
    t0 = time.perf_counter()
    L = solver.power_iteration(gc, sc, iters=20, seed=0)
    _, info = solver.bregman(gc, sc, f, 1e-3, outer=c1.bregman_outer, inner=c1.inner, L=L, prox_iters=50)
    ts = time.perf_counter() - t0
    out["c1_solve"] = {"seconds": ts, "outer": c1.bregman_outer, "inner": c1.inner, "prox_iters": 50,
                       "power_iters": 20, "fista_iterations": sum(i["iterations"] for i in info["inner"]),
                       "cores": threads}
    # the workload's reconstruction on the host: its pair count times the sampled pair time
    out["solve_extrapolated_seconds"] = {"value": 300.0 / v, "note": "about 300 A + A^T pairs (5 x 50 FISTA "
                                         "steps, restarts, 20 power iterations) x the all-core pair time"}
    return out


def unet_experiment(args, g, dev):
    """The U-Net of the learned warm start at the workload's grid: inference and one training step
    (forward, data and weight gradients of its 14 3x3x3 convolutions, the other layers, Adam), CUDA
    events around K runs after W warm-up runs, L2 flushed between runs.  Convolution flops: 2 x 27 x
    cin x cout per voxel for the forward pass, the same again for the data gradient (except the first
    layer's, which is not needed) and for the weight gradient; peak = the measured BF16 tensor rate
    (the dense GEMM burst figure of the machine's cuBLAS measurement)."""
    import torch

    from paper_1605_00133_gb300 import _lib, unet
    net = unet.WarmStartUNet(g.nz, g.ny, g.nx, seed=0)
    gen = torch.Generator(device=dev).manual_seed(1)
    x = torch.randn(g.n, device=dev, generator=gen)
    t = torch.randn(g.n, device=dev, generator=gen)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    fwd = sum(2.0 * 27 * c[0] * c[1] * net.V[c[2]] for c in unet.LAYERS.values())
    dgrad = fwd - 2.0 * 27 * 16 * 16 * net.V[0]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
            flush.fill_(1.0)
        torch.cuda.synchronize()
        total = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        return total / args.steps

    ms_inf = timed(lambda: net.forward(x))
    ms_train = timed(lambda: net.train_step(x, t, lr=1e-5))
    _lib.check(_lib.load().pat_unet_device_status(torch.cuda.current_stream(dev).cuda_stream))
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak = 1910.0
    if os.path.exists(peaks_path):
        peak = float(json.load(open(peaks_path)).get("bf16_tflops", peak))
    return {"grid": [g.nz, g.ny, g.nx], "inference_ms": ms_inf, "train_step_ms": ms_train,
            "conv_gflop_inference": fwd / 1e9, "conv_gflop_train_step": (2 * fwd + dgrad) / 1e9,
            "inference_conv_tflops": fwd / (ms_inf * 1e-3) / 1e12,
            "train_conv_tflops": (2 * fwd + dgrad) / (ms_train * 1e-3) / 1e12,
            "bf16_peak_tflops": peak, "peak_source": "measured bf16_tflops (burst)",
            "note": "whole-step times include the non-convolution layers; the fractions of the peak are "
                    "lower bounds for the convolution kernels alone"}


def warm_start_experiment(args, op, g, dev):
    """Train the U-Net warm start on seeded phantoms of the workload and compare warm vs plain solves
    on held-out phantoms: time to 10 %, 5 % and 2 % relative error against a converged plain
    reconstruction (warmstart.evaluate)."""
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
    train_pairs = warmstart.make_pairs(op, wl, args.warm_train, 1000, lam, wl.bregman_outer,
                                       args.warm_target_inner, L)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    test_pairs = warmstart.make_pairs(op, wl, args.warm_test, 5000, lam, wl.bregman_outer,
                                      args.warm_target_inner, L)
    net = unet.WarmStartUNet(g.nz, g.ny, g.nx, seed=0)
    net.s_in = warmstart.input_scale(train_pairs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = warmstart.train(net, train_pairs, args.warm_epochs, lr=1e-3, seed=0)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    steps = args.warm_epochs * len(train_pairs)
    inners = [10, 25, 50, 100, 200, 300, 450]
    tols = (0.10, 0.05, 0.02)
    ev = warmstart.evaluate(op, net, test_pairs, lam, wl.bregman_outer, inners, L, args.warm_ref_inner, tols)
    op.device_status(dev)

    def med(v):
        v = [x for x in v if x is not None]
        return float(np.median(v)) if len(v) == len(ev) else None
    summary = {}
    for tol in tols:
        k = f"{tol:g}"
        summary[k] = {arm: {"median_seconds": med([e["seconds_to"][k][arm] for e in ev]),
                            "reached": sum(e["seconds_to"][k][arm] is not None for e in ev)}
                      for arm in ("plain", "warm")}
    return {"train_pairs": len(train_pairs), "test_pairs": len(test_pairs), "epochs": args.warm_epochs,
            "target": {"outer": wl.bregman_outer, "inner": args.warm_target_inner, "prox_iters": 50},
            "data_seconds": t_data, "data_seconds_per_pair": t_data / max(len(train_pairs), 1),
            "train_steps": steps, "train_seconds": t_train, "train_ms_per_step": 1e3 * t_train / steps,
            "loss_per_epoch": hist, "L": L, "lambda": lam,
            "reference": {"outer": wl.bregman_outer, "inner": args.warm_ref_inner, "prox_iters": 50},
            "schedule": {"outer": wl.bregman_outer, "inner": inners},
            "network_rel_err": [e["network_rel_err"] for e in ev],
            "target_rel_err": [e["target_rel_err"] for e in ev],
            "inference_seconds": [e["inference_seconds"] for e in ev],
            "seconds_to": summary, "per_phantom": [e["seconds_to"] for e in ev],
            "trajectories": [{"plain": e["plain"], "warm": e["warm"]} for e in ev]}


# sources that do not take part in A or A^T (solver, learned warm start): excluded from the hash
_NOT_OPERATOR = ("pat_solver.cu", "pat_unet.cu", "pat_unet_tc.cu")


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

"""Training and evaluation of the learned warm start (unet.WarmStartUNet) for the TV-Bregman solver.

Data: seeded vessel phantoms of the workload; per phantom the noisy sub-sampled data f = C A p0 + e
(1 % of max|C A p0|), the network input A^T C^T f and the target, a plain TV-Bregman reconstruction
of f (Sec. 4.5-4.6, App. B) with the workload's Bregman steps and `inner_target` FISTA iterations per
step (one solve per phantom; the cost of a target is the data-generation rate).

Evaluation on held-out phantoms, against p_ref = a converged plain TV-Bregman reconstruction (the same
solver and Bregman steps with `inner_ref` FISTA iterations per step, computed once and not timed):
for the plain cold-start solve and for the solve started from the network's output, the wall time
until a reconstruction is within each tolerance (10 %, 5 %, 2 % relative error) of p_ref.  Both arms
run the same schedules with an increasing number of inner iterations per Bregman step (each solve
from scratch, so the timings are of complete solves) and the same step size 1.8/L with L estimated
once per grid; an arm stops once it is within the smallest tolerance.  The warm arm's time includes
the network's inference, and the network's output alone is its first point.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import synth


def make_pairs(op, workload, n: int, seed0: int, lam: float, outer: int, inner_target: int, L: float,
               prox_iters: int = 50):
    """n phantoms (seeds seed0 .. seed0 + n - 1): dicts of device tensors x (input), target, f, p0."""
    out = []
    for i in range(n):
        p0 = torch.tensor(workload.p0(seed_offset=seed0 + i), dtype=torch.float32,
                          device=op.device).reshape(op.image_shape)
        fc = op.forward(p0)
        noise = synth.gaussian_noise(tuple(fc.shape), 0.01 * float(fc.abs().max()), 10_000 + seed0 + i)
        f = fc + torch.tensor(noise, dtype=torch.float32, device=op.device)
        x = op.adjoint(f)
        tgt, _ = op.bregman_solve(f, lam, outer=outer, inner=inner_target, prox_iters=prox_iters, L=L)
        out.append({"x": x.reshape(-1).clone(), "target": tgt.reshape(-1).clone(), "f": f.clone(),
                    "p0": p0.reshape(-1).clone()})
    return out


def input_scale(pairs) -> float:
    """1 / the RMS of the training inputs: network inputs of order one."""
    s = np.mean([float((p["x"] ** 2).mean()) for p in pairs])
    return 1.0 / max(float(np.sqrt(s)), 1e-30)


def train(net, pairs, epochs: int, lr: float, seed: int = 0):
    """Adam on the mean squared error, one pair per step, seeded shuffling; the rate drops by 10 for
    the last quarter of the epochs.  Returns the mean loss of every epoch."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        rate = lr if ep < 0.75 * epochs else 0.1 * lr
        losses = [net.train_step(pairs[i]["x"], pairs[i]["target"], lr=rate).clone()
                  for i in rng.permutation(len(pairs))]
        hist.append(float(torch.stack(losses).mean()))
    return hist


def _timed_solve(op, f, lam, outer, inner, L, warm=None, prox_iters=50):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p, _ = op.bregman_solve(f, lam, outer=outer, inner=inner, prox_iters=prox_iters, L=L, warm=warm)
    torch.cuda.synchronize()
    return p, time.perf_counter() - t0


def evaluate(op, net, pairs, lam: float, outer: int, inners, L: float, inner_ref: int,
             tols=(0.10, 0.05, 0.02), prox_iters: int = 50):
    """Per held-out phantom: p_ref (inner_ref FISTA iterations per Bregman step), both arms'
    (inner iterations, seconds, error vs p_ref) trajectories over `inners`, and each arm's time to
    every tolerance in `tols` (None where its trajectory never gets there)."""
    res = []
    for pr in pairs:
        f = pr["f"]
        p_ref, _ = op.bregman_solve(f, lam, outer=outer, inner=inner_ref, prox_iters=prox_iters, L=L)
        nref = float(p_ref.norm())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        w = net.forward(pr["x"]).reshape(op.image_shape).clone()
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - t0
        e_net = float((w - p_ref).norm()) / nref
        e_tgt = float((pr["target"].reshape(op.image_shape) - p_ref).norm()) / nref
        arms = {"plain": [], "warm": [{"inner": 0, "seconds": t_inf, "rel_err": e_net}]}
        for name in ("plain", "warm"):
            for n in inners:
                if arms[name] and arms[name][-1]["rel_err"] <= min(tols):
                    break
                p, t = _timed_solve(op, f, lam, outer, n, L, warm=w if name == "warm" else None,
                                    prox_iters=prox_iters)
                if name == "warm":
                    t += t_inf
                arms[name].append({"inner": n, "seconds": t, "rel_err": float((p - p_ref).norm()) / nref})

        def first(tr, tol):
            return next((e["seconds"] for e in tr if e["rel_err"] <= tol), None)
        res.append({"network_rel_err": e_net, "target_rel_err": e_tgt, "inference_seconds": t_inf,
                    "plain": arms["plain"], "warm": arms["warm"],
                    "seconds_to": {f"{tol:g}": {"plain": first(arms["plain"], tol),
                                                "warm": first(arms["warm"], tol)} for tol in tols}})
    return res

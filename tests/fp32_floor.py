"""The same k-space recurrence as the FP64 oracle, restated with numpy and scipy.fft in a chosen
precision: the accuracy any FP32 implementation of the scheme can reach (its "FP32 floor").

TEST INFRASTRUCTURE.  It shares no code with the CUDA library or with oracle/pat_oracle.c; it is a
second, independent statement of the discrete model (Sec. 4.3: staggered k-space gradient and
divergence with kappa = sinc(c dt |k| / 2), split-field density, fourth-order PML inside the grid;
A^T as the statement-by-statement transpose run backwards in time, Sec. 4.4), used for three things:

* in float64 it must equal the oracle (tests/test_fp32_floor.py pins it there on small grids);
* in float32 it shows how far an FP32 evaluation of the recurrence lands from the FP64 oracle on
  given data, which is the bar the GPU path is held to where the broadband adjoint cases exceed 1e-5;
* its `round_states` / `round_fft` switches keep either the transforms or the state updates in
  float64 and round only the other to float32, which shows where the FP32 error comes from.

Run as a script it reproduces, on the 64x128x128 / T = 400 workload, the error of the FP32
restatement against the oracle for the data cases the GPU tests use:

    python tests/fp32_floor.py [--T 400] [--cases white,noisy,residual] [--threads N]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np
import scipy.fft as sfft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


class Scheme:
    """Constant tables of one grid: the staggered derivative multipliers on the rfftn half spectrum
    and the PML factors on regular and staggered points, all computed in float64."""

    def __init__(self, g, dtype=np.float32, round_states=True, round_fft=True, workers=-1):
        self.g = g
        self.rdt = np.dtype(dtype)
        self.cdt = np.result_type(self.rdt, np.complex64)
        self.round_states = round_states
        self.round_fft = round_fft
        self.workers = workers
        nz, ny, nx = g.nz, g.ny, g.nx

        def wn(n, half=False):
            m = np.arange(n // 2 + 1) if half else np.arange(n)
            mm = np.where(m < n // 2, m, m - n)  # the Nyquist bin n/2 taken negative
            return 2 * np.pi * mm / (n * g.dx)

        kz = wn(nz)[:, None, None]
        ky = wn(ny)[None, :, None]
        kx = wn(nx, half=True)[None, None, :]
        kabs = np.sqrt(kz ** 2 + ky ** 2 + kx ** 2)
        xk = 0.5 * g.c * g.dt * kabs
        with np.errstate(invalid="ignore", divide="ignore"):
            kappa = np.where(xk == 0, 1.0, np.sin(xk) / np.where(xk == 0, 1.0, xk))
        self.mult = {}
        for axis, k in enumerate((kz, ky, kx)):
            for s in (+1, -1):
                m = 1j * k * kappa * np.exp(1j * s * k * g.dx / 2)
                self.mult[(axis, s)] = np.broadcast_to(m, kappa.shape)

        def pml(n, staggered):
            P = g.pml_size
            pos = np.arange(n) + (0.5 if staggered else 0.0)
            if P <= 0:
                return np.ones(n)
            d = np.where(pos < P, P - pos, np.where(pos > n - 1 - P, pos - (n - 1 - P), 0.0))
            alpha = g.pml_alpha * (g.c / g.dx) * (d / P) ** 4
            return np.exp(-alpha * g.dt / 2)

        shapes = [(nz, 1, 1), (1, ny, 1), (1, 1, nx)]
        self.a = [pml(n, False).reshape(sh) for n, sh in zip((nz, ny, nx), shapes)]
        self.as_ = [pml(n, True).reshape(sh) for n, sh in zip((nz, ny, nx), shapes)]

    # precision of a transform and of a state update
    def _f(self, x):
        return x.astype(self.rdt if self.round_fft else np.float64, copy=False)

    def _s(self, x):
        return x.astype(self.rdt if self.round_states else np.float64, copy=False)

    def deriv(self, f, axis, s, transpose=False):
        """Re F^-1[ m F f ], m = i k_axis kappa exp(s i k_axis dx / 2) (conjugated for the transpose)."""
        g = self.g
        m = self.mult[(axis, s)]
        if transpose:
            m = np.conj(m)
        ct = self.cdt if self.round_fft else np.complex128
        spec = sfft.rfftn(self._f(f), workers=self.workers)
        spec = (spec * m.astype(ct)).astype(ct, copy=False)
        return sfft.irfftn(spec, s=(g.nz, g.ny, g.nx), workers=self.workers)

    def forward_plane(self, p0):
        """pbar[n] = p^n on the plane z = sensor_z, n = 0..T-1 (the oracle's or_forward)."""
        g = self.g
        c2, dt, rho0 = g.c * g.c, g.dt, g.rho0
        zs = g.sensor_z
        p0 = self._s(np.asarray(p0, np.float64))
        rho = [self._s(p0 / (3 * c2)) for _ in range(3)]
        u = [self._s(dt / (2 * rho0) * self.deriv(p0, i, +1)) for i in range(3)]
        out = np.zeros((g.T, g.ny * g.nx))
        out[0] = p0[zs].ravel()
        for n in range(g.T - 1):
            p = self._s(c2 * (rho[0] + rho[1] + rho[2]))
            for i in range(3):
                u[i] = self._s(self.as_[i] * (self.as_[i] * u[i] - dt / rho0 * self.deriv(p, i, +1)))
            for i in range(3):
                rho[i] = self._s(self.a[i] * (self.a[i] * rho[i] - dt * rho0 * self.deriv(u[i], i, -1)))
            out[n + 1] = (c2 * (rho[0][zs] + rho[1][zs] + rho[2][zs])).ravel()
        return out

    def adjoint_plane(self, y):
        """A^T of forward_plane: the data enter as a source at every step (the oracle's or_adjoint)."""
        g = self.g
        c2, dt, rho0 = g.c * g.c, g.dt, g.rho0
        zs = g.sensor_z
        y = np.asarray(y, np.float64).reshape(g.T, g.ny, g.nx)
        shape = (g.nz, g.ny, g.nx)
        lr = [self._s(np.zeros(shape)) for _ in range(3)]
        lu = [self._s(np.zeros(shape)) for _ in range(3)]
        for n in range(g.T - 1, 0, -1):
            for i in range(3):
                lr[i] = lr[i].copy()
                lr[i][zs] += c2 * y[n]
                lr[i] = self._s(lr[i])
            for i in range(3):
                t = self.deriv(self.a[i] * lr[i], i, -1, transpose=True)
                lu[i] = self._s(lu[i] - dt * rho0 * t)
                lr[i] = self._s(self.a[i] * self.a[i] * lr[i])
            lp = np.zeros(shape)
            for i in range(3):
                t = self.deriv(self.as_[i] * lu[i], i, +1, transpose=True)
                lp = self._s(lp - dt / rho0 * t)
                lu[i] = self._s(self.as_[i] * self.as_[i] * lu[i])
            for i in range(3):
                lr[i] = self._s(lr[i] + c2 * lp)
        p = np.zeros(shape)
        p[zs] += y[0]
        for i in range(3):
            p = self._s(p + lr[i] / (3 * c2) + dt / (2 * rho0) * self.deriv(lu[i], i, +1, transpose=True))
        return p


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _cases(w, T, names, oracle):
    """Full-plane data of the 64x128x128 workload: white noise, A p0 + 1 % noise, and a residual
    A p - f of a solver iterate p (the back-projection of the noisy data, scaled by the step of a
    gradient iteration from zero), each as the workloads' tests build them."""
    from paper_1605_00133_gb300 import presets, synth
    g = presets.Grid(w.grid.nz, w.grid.ny, w.grid.nx, dx=w.grid.dx, T=T, pml_size=w.grid.pml_size)
    out = {}
    if "white" in names:
        out["white"] = np.random.default_rng(0).standard_normal((T, g.m_plane))
    if "noisy" in names or "residual" in names:
        f = oracle.forward_plane(g, w.p0())
        fn = synth.add_relative_noise(f, 0.01, 4)
        if "noisy" in names:
            out["noisy"] = fn
        if "residual" in names:
            b = oracle.adjoint_plane(g, fn)
            Ab = oracle.forward_plane(g, b)
            step = float(np.sum(fn * Ab) / np.sum(Ab * Ab))  # exact line search along A^T f
            out["residual"] = step * Ab - fn
    return g, out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--T", type=int, default=400)
    ap.add_argument("--cases", default="white,noisy,residual")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--variants", action="store_true",
                    help="also run with only the transforms, or only the state updates, in float32")
    args = ap.parse_args()
    import oracle
    from paper_1605_00133_gb300 import presets
    if args.threads:
        oracle.set_threads(args.threads)
    w = presets.workload("c2")
    g, cases = _cases(w, args.T, args.cases.split(","), oracle)
    variants = [("fp32", True, True)]
    if args.variants:
        variants += [("fp32 transforms only", False, True), ("fp32 states only", True, False)]
    for name, y in cases.items():
        t0 = time.time()
        ref = oracle.adjoint_plane(g, y)
        for vname, rs, rf in variants:
            sc = Scheme(g, np.float32, round_states=rs, round_fft=rf)
            e = rel(sc.adjoint_plane(y), ref)
            print(f"adjoint, {name:8s} T={args.T}: {vname:22s} rel-L2 vs FP64 oracle {e:.3e}"
                  f"  ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    main()

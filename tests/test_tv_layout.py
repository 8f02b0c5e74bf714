"""Host-side model of the TV prox kernel's tiling (tv_step_kernel in pat_solver.cu), no GPU.

The kernel runs one primal-dual iteration per launch: a CTA of 9 warps owns a 32 x 8 tile of (x, y)
columns over a run of z planes (lanes = x, warps = y, warp 0 the halo row y0 - 1), exchanges x
neighbours by warp shuffle (lane 31 reads x0 + 32 itself, lane 0 of an output row also evaluates
the dual at x0 - 1), y neighbours through shared memory, keeps the z predecessor's new dual in a
register, and evaluates the plane before its run without storing it.  This test restates the
per-thread reads, the shuffles, the two shared-memory exchanges and the stores of that schedule in
FP64 and checks, over ragged shapes, batches and several runs and x tiles, that every read is inside
its buffer, every voxel is written exactly once, and the iterates equal the oracle's prox (App. B).
"""
import math

import numpy as np
import pytest

ROWS = 8            # output rows of a CTA
WARPS = ROWS + 1    # plus the halo row


def runs(nz, gx, gy, B):
    cols = gx * gy * B
    nruns = max(1, min((512 + cols - 1) // cols, (nz + 3) // 4))
    zrun = (nz + nruns - 1) // nruns
    return zrun, (nz + zrun - 1) // zrun


class Reads:
    """A buffer whose every read is checked against its bounds."""
    def __init__(self, a):
        self.a = a

    def __getitem__(self, i):
        assert 0 <= i < len(self.a), (i, len(self.a))
        return self.a[i]


def project(a, b, e, alpha):
    n = math.sqrt(a * a + b * b + e * e)
    s = alpha / n if n > alpha else 1.0
    return a * s, b * s, e * s


def step(qb_in, xi_in, q, p, sigma, alpha, tau, theta, nz, ny, nx, B):
    """One launch: returns qbar and xi of the next iteration (q is updated in place)."""
    n, N = nz * ny * nx, B * nz * ny * nx
    gx, gy = (nx + 31) // 32, (ny + ROWS - 1) // ROWS
    zrun, nruns = runs(nz, gx, gy, B)
    qb, xi, qr, pr = Reads(qb_in), Reads(xi_in), Reads(q.copy()), Reads(p)
    qb_out, xi_out = np.full(N, np.nan), np.full(3 * N, np.nan)
    written = np.zeros(N, int)
    plane = ny * nx
    for bz in range(B * nruns):
        b, run = divmod(bz, nruns)
        z0 = run * zrun
        z1 = min(z0 + zrun, nz)
        for bx in range(gx):
            for by in range(gy):
                x0 = 32 * bx
                T = {}
                for w in range(WARPS):
                    for lane in range(32):
                        x, y = x0 + lane, by * ROWS - 1 + w
                        yin = 0 <= y < ny
                        T[w, lane] = dict(x=x, y=y, inn=yin and x < nx, own=yin and x < nx and w > 0,
                                          xn=x + 1 < nx, yn=y + 1 < ny, base=b * n + y * nx + x,
                                          halo=lane == 0 and x0 > 0 and yin and w > 0,
                                          right=lane == 31 and x0 + 32 < nx and yin,
                                          down=w == WARPS - 1 and yin and x < nx and y + 1 < ny)
                zs = z0 - 1 if z0 > 0 else z0
                for t in T.values():
                    t["qc"] = qb[t["base"] + zs * plane] if t["inn"] else 0.0
                    t["qlc"] = qb[t["base"] - 1 + zs * plane] if t["halo"] else 0.0
                    t["pz"] = 0.0
                for z in range(zs, z1):
                    zn = z + 1 < nz
                    sq = np.zeros((WARPS, 32))
                    sy = np.zeros((WARPS, 32))
                    for (w, lane), t in T.items():  # this plane's reads
                        o = t["base"] + z * plane
                        t["store"] = t["own"] and z >= z0
                        t["qn"] = qb[o + plane] if t["inn"] and zn else 0.0
                        t["xz"], t["xy"], t["xx"] = (xi[o], xi[N + o], xi[2 * N + o]) if t["inn"] else (0.0,) * 3
                        t["qv"] = qr[o] if t["store"] else 0.0
                        t["pv"] = pr[o] if t["store"] else 0.0
                        t["qr"] = qb[o + 1] if t["right"] else 0.0
                        t["qd"] = qb[o + nx] if t["down"] else 0.0
                        h = t["halo"]
                        t["qln"] = qb[o - 1 + plane] if h and zn else 0.0
                        t["qld"] = qb[o - 1 + nx] if h and t["yn"] else 0.0
                        t["l"] = (xi[o - 1], xi[N + o - 1], xi[2 * N + o - 1]) if h else (0.0,) * 3
                        sq[w, lane] = t["qc"]
                    for (w, lane), t in T.items():  # new dual (and, lane 0, the one at x0 - 1)
                        qxn = T[w, lane + 1]["qc"] if lane < 31 else t["qc"]  # shuffle down by 1
                        qyn = sq[w + 1, lane] if w < WARPS - 1 else t["qd"]
                        gz = t["qn"] - t["qc"] if zn else 0.0
                        gy_ = qyn - t["qc"] if t["yn"] else 0.0
                        gx_ = ((qxn if lane < 31 else t["qr"]) - t["qc"]) if t["xn"] else 0.0
                        t["d"] = project(t["xz"] + sigma * gz, t["xy"] + sigma * gy_, t["xx"] + sigma * gx_, alpha)
                        t["dlx"] = 0.0
                        if t["halo"]:
                            lz, ly, lx = t["l"]
                            t["dlx"] = project(lz + sigma * ((t["qln"] - t["qlc"]) if zn else 0.0),
                                               ly + sigma * ((t["qld"] - t["qlc"]) if t["yn"] else 0.0),
                                               lx + sigma * (t["qc"] - t["qlc"]), alpha)[2]
                        sy[w, lane] = t["d"][1]
                    for (w, lane), t in T.items():  # primal step and stores
                        dz, dy, dx = t["d"]
                        dxl = T[w, lane - 1]["d"][2] if lane > 0 else dx  # shuffle up by 1
                        if t["store"]:
                            o = t["base"] + z * plane
                            gt = 0.0
                            if zn:
                                gt -= dz
                            if z > 0:
                                gt += t["pz"]
                            if t["yn"]:
                                gt -= dy
                            if t["y"] > 0:
                                gt += sy[w - 1, lane]
                            if t["xn"]:
                                gt -= dx
                            if t["x"] > 0:
                                gt += dxl if lane > 0 else t["dlx"]
                            qnew = max(0.0, (-tau * gt + (tau * t["pv"] + t["qv"])) / (1.0 + tau))
                            q[o] = qnew
                            qb_out[o] = theta * (qnew - t["qv"]) + qnew
                            xi_out[o], xi_out[N + o], xi_out[2 * N + o] = dz, dy, dx
                            written[o] += 1
                    for t in T.values():
                        t["pz"], t["qc"], t["qlc"] = t["d"][0], t["qn"], t["qln"]
    assert (written == 1).all(), np.unique(written, return_counts=True)
    return qb_out, xi_out


@pytest.mark.parametrize("shape,B", [((5, 9, 33), 1), ((9, 17, 40), 2), ((6, 1, 1), 1), ((4, 20, 1), 1),
                                     ((13, 10, 64), 1)])
def test_tiling_matches_the_oracle_prox(shape, B, oracle_mod):
    from oracle import solver
    nz, ny, nx = shape
    n = nz * ny * nx
    P = np.random.default_rng(3).standard_normal((B,) + shape) * 0.5 + 0.2
    p = P.ravel().copy()
    q = np.maximum(0.0, p)
    qb, xi = q.copy(), np.zeros(3 * B * n)
    alpha, iters = 0.2, 5
    tau = 1.0 / math.sqrt(12.0)
    sigma = 1.0 / (tau * 12.0)
    for _ in range(iters):
        theta = 1.0 / math.sqrt(1.0 + 2.0 * tau)
        qb, xi = step(qb, xi, q, p, sigma, alpha, tau, theta, nz, ny, nx, B)
        tau, sigma = theta * tau, sigma / theta
    for b in range(B):
        ref = solver.tv_prox(P[b], alpha, iters)
        got = q[b * n:(b + 1) * n].reshape(shape)
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)

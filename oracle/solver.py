"""FP64 oracle for the variational reconstruction of arXiv:1605.00133 (TEST INFRASTRUCTURE ONLY).

Plain numpy, double precision, written in the paper's order:
  tv, grad, grad_T     discrete isotropic TV with forward differences and Neumann boundary (App. A)
  tv_prox              positivity-constrained TV denoising, argmin_{q>=0} 1/2||q-p||^2 + alpha TV(q)
                       (Eq. TV+Denoise, App. B), by the primal-dual hybrid gradient method the paper
                       names (Chambolle-Pock, accelerated variant for a strongly convex primal term),
                       with the duality gap as certificate
  power_iteration      L ~ ||A^T C^T C A||_2 (App. B)
  fista                accelerated proximal gradient with restart and up to 5 backtracking steps,
                       eta = 1.8 / L (Eq. ProxGradDesc and the bullet list after it, App. B)
  bregman              Bregman iterations (Eqs. BregIterA/B, Sec. 4.6), b^0 = 0
The forward and adjoint operators are the oracle's own (`oracle.forward`, `oracle.adjoint`).
"""
from __future__ import annotations

import math

import numpy as np

from . import adjoint as _adjoint
from . import forward as _forward

L2_GRAD = 12.0  # ||grad||^2 <= 4 * 3 for forward differences in 3D


# --------------------------------------------------------------------------------- TV (App. A)

def grad(q):
    """Forward differences along z, y, x; the difference beyond the last voxel is zero (Neumann)."""
    q = np.asarray(q, np.float64)
    g = np.zeros((3,) + q.shape)
    g[0, :-1] = q[1:] - q[:-1]
    g[1, :, :-1] = q[:, 1:] - q[:, :-1]
    g[2, :, :, :-1] = q[:, :, 1:] - q[:, :, :-1]
    return g


def grad_T(xi):
    """Exact transpose of `grad` (the negative divergence)."""
    out = np.zeros(xi.shape[1:])
    out[:-1] -= xi[0, :-1]
    out[1:] += xi[0, :-1]
    out[:, :-1] -= xi[1, :, :-1]
    out[:, 1:] += xi[1, :, :-1]
    out[:, :, :-1] -= xi[2, :, :, :-1]
    out[:, :, 1:] += xi[2, :, :, :-1]
    return out


def tv(q):
    """TV(q) = sum over voxels of the Euclidean norm of the forward-difference gradient."""
    return float(np.sum(np.sqrt(np.sum(grad(q) ** 2, axis=0))))


def project_balls(xi, radius):
    """Pointwise projection of the 3-vectors xi[:, v] onto the ball of the given radius."""
    nrm = np.sqrt(np.sum(xi ** 2, axis=0))
    return xi / np.maximum(1.0, nrm / radius)[None] if radius > 0 else np.zeros_like(xi)


# --------------------------------------------------------------------------------- TV prox (App. B)

def tv_prox_gap(q, xi, p, alpha):
    """Duality gap of min_{q>=0} 1/2||q-p||^2 + alpha TV(q) at primal q, dual xi (||xi_v|| <= alpha).
    Dual value D(xi) = min_{q>=0} 1/2||q-p||^2 + <q, grad^T xi>, attained at max(0, p - grad^T xi)."""
    primal = 0.5 * np.sum((q - p) ** 2) + alpha * tv(q)
    gt = grad_T(xi)
    qd = np.maximum(0.0, p - gt)
    dual = 0.5 * np.sum((qd - p) ** 2) + np.sum(qd * gt)
    return primal - dual


def pdhg_schedule(iters, tau0=None, gamma=1.0):
    """Step sizes (tau_n, sigma_n, theta_n) of the accelerated primal-dual method for a
    gamma-strongly convex primal term: theta_n = 1/sqrt(1 + 2 gamma tau_n), tau_{n+1} = theta_n
    tau_n, sigma_{n+1} = sigma_n / theta_n, with tau_0 sigma_0 ||grad||^2 = 1."""
    tau = tau0 if tau0 is not None else 1.0 / math.sqrt(L2_GRAD)
    sigma = 1.0 / (tau * L2_GRAD)
    out = []
    for _ in range(iters):
        theta = 1.0 / math.sqrt(1.0 + 2.0 * gamma * tau)
        out.append((tau, sigma, theta))
        tau, sigma = theta * tau, sigma / theta
    return out


def tv_prox(p, alpha, iters=200, nonneg=True, return_dual=False):
    """argmin_{q >= 0} 1/2 ||q - p||^2 + alpha TV(q) by the primal-dual hybrid gradient method:
        xi    <- project_{||.|| <= alpha}(xi + sigma grad(qbar))
        q_new <- max(0, (q - tau grad^T(xi) + tau p) / (1 + tau))
        qbar  <- q_new + theta (q_new - q)
    starting from q = qbar = max(0, p), xi = 0."""
    p = np.asarray(p, np.float64)
    clip = (lambda v: np.maximum(0.0, v)) if nonneg else (lambda v: v)
    q = clip(p.copy())
    qbar = q.copy()
    xi = np.zeros((3,) + p.shape)
    if alpha <= 0:
        return (q, xi) if return_dual else q
    for tau, sigma, theta in pdhg_schedule(iters):
        xi = project_balls(xi + sigma * grad(qbar), alpha)
        q_new = clip((q - tau * grad_T(xi) + tau * p) / (1.0 + tau))
        qbar = q_new + theta * (q_new - q)
        q = q_new
    return (q, xi) if return_dual else q


# --------------------------------------------------------------------------------- solver (App. B, Sec. 4.6)

def power_iteration(g, s, iters=20, seed=0, x0=None):
    """L ~ ||A^T C^T C A||_2 by power iteration from x0 (default: a seeded Gaussian start)."""
    x = np.random.default_rng(seed).standard_normal(g.shape) if x0 is None else np.array(x0, np.float64)
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = _adjoint(g, s, _forward(g, s, x))
        lam = float(np.linalg.norm(y))
        x = y / lam
    return lam


def objective(Ax, data, x, lam):
    return 0.5 * float(np.sum((Ax - data) ** 2)) + lam * tv(x)


def fista(g, s, data, lam, x0, L, iters, prox_iters=200, eta_scale=1.8, restart=True,
          max_backtrack=5, stall=5):
    """Accelerated proximal gradient for min_{x>=0} 1/2 ||C A x - data||^2 + lam TV(x):
        x_j = prox_{eta lam}(y_j - eta A^T C^T (C A y_j - data)),  eta = eta_scale / L,
        y_{j+1} = x_j + (t_j - 1)/t_{j+1} (x_j - x_{j-1}),  t_{j+1} = (1 + sqrt(1 + 4 t_j^2)) / 2.
    If the energy increases, the momentum restarts and the iterate becomes a plain gradient step from
    x_{j-1}, with eta halved up to max_backtrack times for that iteration only.  Stops early when x
    does not change or min E has not decreased `stall` times in a row.  C A y_j is formed from the
    stored C A x_j, C A x_{j-1} by linearity.  Returns (x, C A x, info)."""
    eta = eta_scale / L
    x_prev = np.asarray(x0, np.float64).copy()
    Ax_prev = _forward(g, s, x_prev)
    E_prev = objective(Ax_prev, data, x_prev, lam)
    y, Ay = x_prev.copy(), Ax_prev.copy()
    t = 1.0
    best, since_best = E_prev, 0
    info = {"energies": [E_prev], "restarts": 0, "iterations": 0}
    for _ in range(iters):
        gradient = _adjoint(g, s, Ay - data)
        x = tv_prox(y - eta * gradient, eta * lam, prox_iters)
        Ax = _forward(g, s, x)
        E = objective(Ax, data, x, lam)
        if restart and E > E_prev:
            info["restarts"] += 1
            t = 1.0
            gradient = _adjoint(g, s, Ax_prev - data)
            eta_b = eta
            for _b in range(max_backtrack + 1):
                x = tv_prox(x_prev - eta_b * gradient, eta_b * lam, prox_iters)
                Ax = _forward(g, s, x)
                E = objective(Ax, data, x, lam)
                if E <= E_prev:
                    break
                eta_b *= 0.5
            if E > E_prev:  # no descent found: keep the previous iterate
                x, Ax, E = x_prev.copy(), Ax_prev.copy(), E_prev
        info["iterations"] += 1
        info["energies"].append(E)
        unchanged = np.array_equal(x, x_prev)
        t_next = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        beta = (t - 1.0) / t_next
        y = x + beta * (x - x_prev)
        Ay = Ax + beta * (Ax - Ax_prev)
        x_prev, Ax_prev, E_prev, t = x, Ax, E, t_next
        if E < best:
            best, since_best = E, 0
        else:
            since_best += 1
        if unchanged or since_best >= stall:
            break
    return x_prev, Ax_prev, info


def bregman(g, s, f, lam, outer, inner, L=None, x0=None, prox_iters=200, **kw):
    """Bregman iterations (Eqs. BregIterA/B): p^{k+1} = argmin 1/2||C A p - (f + b^k)||^2 + lam TV+(p),
    b^{k+1} = b^k + (f - C A p^{k+1}), b^0 = 0; each subproblem solved by `fista`, warm-started
    from p^k.  Returns (p, info) with the data residual ||C A p^k - f|| after every outer step."""
    f = np.asarray(f, np.float64)
    if L is None:
        L = power_iteration(g, s)
    p = np.zeros(g.shape) if x0 is None else np.asarray(x0, np.float64).copy()
    b = np.zeros_like(f)
    info = {"L": L, "residuals": [], "inner": []}
    for _ in range(outer):
        p, Ap, fi = fista(g, s, f + b, lam, p, L, inner, prox_iters=prox_iters, **kw)
        b = b + (f - Ap)
        info["residuals"].append(float(np.linalg.norm(Ap - f)))
        info["inner"].append(fi)
    return p, info

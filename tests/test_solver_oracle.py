"""Pins of the FP64 solver oracle (TV, TV prox, FISTA, Bregman) against facts fixed outside it."""
import numpy as np
import pytest

from paper_1605_00133_gb300 import presets, synth


@pytest.fixture(scope="module")
def sol(oracle_mod):
    from oracle import solver
    return solver


def test_grad_transpose_is_exact(sol):
    rng = np.random.default_rng(0)
    q = rng.standard_normal((5, 6, 7))
    xi = rng.standard_normal((3, 5, 6, 7))
    assert abs(np.sum(sol.grad(q) * xi) - np.sum(q * sol.grad_T(xi))) < 1e-12


def test_tv_closed_forms(sol):
    assert sol.tv(np.full((4, 5, 6), 3.0)) == 0.0
    q = np.zeros((4, 5, 6))
    q[:, :, 3:] = 2.0           # a jump of 2 across a 4x5 face
    assert sol.tv(q) == pytest.approx(2.0 * 4 * 5)
    q = np.zeros((1, 1, 4))
    q[0, 0] = [0, 3, 4, 4]      # 1D: sum of |differences| (App. A, isotropic = absolute in 1D)
    assert sol.tv(q) == pytest.approx(4.0)
    # isotropic: a voxel with unit differences along two axes contributes sqrt(2)
    q = np.zeros((1, 2, 2))
    q[0, 0, 1] = 1.0
    q[0, 1, 0] = 1.0
    assert sol.tv(q) == pytest.approx(np.sqrt(2.0) + 1.0 + 1.0)


def test_prox_of_constant_nonnegative_image_is_itself(sol):
    p = np.full((6, 5, 4), 0.7)
    assert np.abs(sol.tv_prox(p, 0.3, 50) - p).max() < 1e-12


def test_prox_alpha_zero_is_clipping(sol):
    p = np.random.default_rng(1).standard_normal((4, 4, 4))
    assert np.array_equal(sol.tv_prox(p, 0.0), np.maximum(0, p))


def test_prox_large_alpha_gives_clipped_mean(sol):
    """For alpha beyond the data's total variation scale the minimiser is the constant max(0, mean p)."""
    rng = np.random.default_rng(2)
    p = 0.3 + 0.1 * rng.standard_normal((6, 6, 6))
    q = sol.tv_prox(p, 50.0, 1500)
    assert np.abs(q - max(0.0, p.mean())).max() < 1e-4


def test_prox_duality_gap_certifies_optimality(sol):
    rng = np.random.default_rng(3)
    p = rng.standard_normal((8, 8, 8))
    gaps = []
    for alpha in (0.05, 0.5):
        for iters in (500, 4000):
            q, xi = sol.tv_prox(p, alpha, iters, return_dual=True)
            gaps.append(sol.tv_prox_gap(q, xi, p, alpha) / (0.5 * np.sum(p ** 2)))
    assert min(gaps) >= -1e-12
    # accelerated rate: the gap falls roughly like 1/n^2 (measured 2.4e-7 -> 3.6e-9, 1.1e-5 -> 1.6e-7)
    assert gaps[1] < 1e-8 and gaps[3] < 1e-6
    assert gaps[1] < gaps[0] / 20 and gaps[3] < gaps[2] / 20


def test_prox_of_a_1d_signal_matches_exact_dual_qp(sol):
    """An image that varies along x only reduces to 1D TV denoising scaled by the face size.  For a
    nonnegative input the 1D solution stays within the input's range, so the constraint is inactive,
    and the exact solution is p - D^T u with u = argmin_{|u| <= alpha} 1/2 ||p - D^T u||^2 (bounded
    least squares, solved by scipy)."""
    lsq_linear = pytest.importorskip("scipy.optimize").lsq_linear
    rng = np.random.default_rng(4)
    n = 24
    line = np.abs(np.cumsum(rng.standard_normal(n))) + 0.5
    alpha = 0.4
    D = np.zeros((n - 1, n))
    D[np.arange(n - 1), np.arange(n - 1)] = -1.0
    D[np.arange(n - 1), np.arange(1, n)] = 1.0
    res = lsq_linear(D.T, line, bounds=(-alpha, alpha), lsmr_tol="auto", tol=1e-14, max_iter=10000)
    exact = line - D.T @ res.x
    img = np.broadcast_to(line, (3, 4, n)).copy()
    q = sol.tv_prox(img, alpha, 3000)

    def obj(v):
        return 0.5 * np.sum((v - line) ** 2) + alpha * np.sum(np.abs(np.diff(v)))
    # the primal-dual iterate approaches the minimiser like 1/n (5e-4 after 3000 steps) and its
    # objective like 1/n^2
    assert np.abs(q - exact[None, None, :]).max() < 1e-3
    for row in q.reshape(-1, n):
        assert abs(obj(row) - obj(exact)) < 1e-6 * obj(exact)


def test_power_iteration_matches_dense_svd(oracle_mod, sol):
    g = presets.Grid(8, 8, 8, T=8, pml_size=2)
    s = presets.make_sampling(g, presets.KIND_RSP, 20, 0)
    N = g.n
    A = np.empty((g.T * s.m, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        A[:, j] = oracle_mod.forward(g, s, e.reshape(g.shape)).ravel()
    smax = np.linalg.svd(A, compute_uv=False)[0]
    L = sol.power_iteration(g, s, iters=200, seed=1)
    assert L == pytest.approx(smax ** 2, rel=1e-6)


@pytest.fixture(scope="module")
def small_problem(oracle_mod):
    g = presets.Grid(16, 16, 16, T=24, pml_size=3)
    s = presets.make_sampling(g, presets.KIND_RSP, 64, 5)
    p_true = synth.gaussian_balls(g.shape, 2, 1.5, 6, pml=3)
    f = synth.add_relative_noise(oracle_mod.forward(g, s, p_true), 0.01, 7)
    return g, s, p_true, f


def test_fista_energy_never_increases(small_problem, sol):
    g, s, p_true, f = small_problem
    L = sol.power_iteration(g, s, iters=30)
    x, Ax, info = sol.fista(g, s, f, 1e-3, np.zeros(g.shape), L, 25, prox_iters=100)
    E = np.array(info["energies"])
    assert np.all(np.diff(E) <= 1e-12 * E[0])
    assert x.min() >= 0


def test_bregman_residual_decreases(small_problem, sol):
    """The data residual ||C A p^k - f|| of the Bregman iterates decreases monotonically (Sec. 4.6)."""
    g, s, p_true, f = small_problem
    p, info = sol.bregman(g, s, f, 5e-3, outer=4, inner=15, prox_iters=100)
    r = np.array(info["residuals"])
    assert np.all(np.diff(r) <= 1e-9 * r[0]), r
    assert p.min() >= 0

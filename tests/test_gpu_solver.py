"""GPU parity of the TV prox and the FISTA + Bregman solver against the FP64 oracle (through the C ABI).

The GPU and the oracle run the same iterations with the same step schedules, so the comparison is
iterate against iterate: FP32 fields against FP64.  Tolerances: the prox at a fixed iteration
count within 1e-5 relative L2; the full solver within 1e-4 (dozens of FP32 A/A^T applications and
prox calls chained, each within 1e-5).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1605_00133_gb300 import presets, synth  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda", 0)


@pytest.fixture(scope="module")
def sol(oracle_mod):
    from oracle import solver
    return solver


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def op_for(g, s):
    from paper_1605_00133_gb300.operators import PatOperator
    return PatOperator(g, s)


@pytest.mark.parametrize("shape,batch,alpha,iters", [
    ((32, 32, 32), 1, 0.05, 100), ((16, 32, 8), 1, 0.3, 300), ((64, 128, 128), 1, 0.02, 50),
    # lines shorter than a warp, batches, many runs of z planes, several x tiles of 32
    ((8, 16, 16), 2, 0.1, 60), ((256, 8, 8), 1, 0.1, 40), ((8, 8, 256), 1, 0.1, 40)])
def test_tv_prox_matches_oracle(dev, sol, shape, batch, alpha, iters):
    """The fused primal-dual kernel (one launch per iteration: z-marching CTAs of 32 x 8 columns,
    warp-shuffle x neighbours, a halo row and column, runs of z planes) against the oracle's prox."""
    g = presets.Grid(*shape, T=2, pml_size=1, batch=batch)
    op = op_for(g, presets.Sampling(presets.KIND_FULL, g.m_plane))
    p = np.random.default_rng(1).standard_normal((batch,) + shape) * 0.5 + 0.2
    x = torch.tensor(p, dtype=torch.float32, device=dev).reshape(op.image_shape)
    got = op.tv_prox(x, alpha, iters).double().cpu().numpy().reshape((batch,) + shape)
    for b in range(batch):
        ref = sol.tv_prox(p[b], alpha, iters)
        assert rel(got[b], ref) < 1e-5
    assert got.min() >= 0


def test_tv_prox_special_cases_and_aliasing(dev):
    g = presets.Grid(16, 16, 16, T=2, pml_size=1, batch=2)
    op = op_for(g, presets.Sampling(presets.KIND_FULL, g.m_plane))
    const = torch.full(op.image_shape, 0.7, device=dev)
    assert float((op.tv_prox(const, 0.3, 50) - const).abs().max()) < 1e-6
    p = torch.randn(op.image_shape, device=dev)
    assert torch.equal(op.tv_prox(p, 0.0, 10), p.clamp_min(0))
    a = op.tv_prox(p, 0.1, 40)
    q = p.clone()
    op.tv_prox(q, 0.1, 40, out=q)  # in place
    assert float((a - q).abs().max()) == 0.0


@pytest.fixture(scope="module")
def c1_problem(oracle_mod):
    w = presets.workload("c1")
    g, s = w.grid, w.sampling
    p_true = w.p0()
    f = synth.add_relative_noise(oracle_mod.forward(g, s, p_true), 0.01, 4)
    return g, s, p_true, f


def test_bregman_solve_matches_oracle(dev, sol, c1_problem):
    """32^3, T = 64, rSP 25 %: 2 Bregman steps x 8 FISTA iterations, 40 prox iterations, the oracle's L."""
    g, s, p_true, f = c1_problem
    L = sol.power_iteration(g, s, iters=20, seed=0)
    lam = 1e-3
    p_ref, info = sol.bregman(g, s, f, lam, outer=2, inner=8, L=L, prox_iters=40)
    op = op_for(g, s)
    ft = torch.tensor(f, dtype=torch.float32, device=dev).reshape(op.data_shape)
    p, rep = op.bregman_solve(ft, lam, outer=2, inner=8, prox_iters=40, L=L)
    got = p.double().cpu().numpy().reshape(g.shape)
    assert rep["restarts"] == sum(i["restarts"] for i in info["inner"])
    assert rep["inner_total"] == sum(i["iterations"] for i in info["inner"])
    assert rel(got, p_ref) < 1e-4
    np.testing.assert_allclose(rep["residuals"], info["residuals"], rtol=1e-4)


@pytest.mark.slow
def test_bregman_solve_on_the_c2_grid_matches_oracle(dev, sol, oracle_mod):
    """The headline grid and sampling (64x128x128, 10-voxel PML, rSP 2048 of 16384, vessel phantom)
    at T = 16: 2 Bregman steps x 4 FISTA iterations, 20 prox iterations, L from 5 oracle power
    iterations; iterate for iterate against the FP64 oracle like the 32^3 case."""
    w = presets.shrink(presets.workload("c2"), 16)
    g, s = w.grid, w.sampling
    f = synth.add_relative_noise(oracle_mod.forward(g, s, w.p0()), 0.01, 4)
    L = sol.power_iteration(g, s, iters=5, seed=0)
    lam = 2e-4
    p_ref, info = sol.bregman(g, s, f, lam, outer=2, inner=4, L=L, prox_iters=20)
    op = op_for(g, s)
    ft = torch.tensor(f, dtype=torch.float32, device=dev).reshape(op.data_shape)
    p, rep = op.bregman_solve(ft, lam, outer=2, inner=4, prox_iters=20, L=L)
    got = p.double().cpu().numpy().reshape(g.shape)
    assert rep["restarts"] == sum(i["restarts"] for i in info["inner"])
    assert rep["inner_total"] == sum(i["iterations"] for i in info["inner"])
    assert rel(got, p_ref) < 1e-4
    np.testing.assert_allclose(rep["residuals"], info["residuals"], rtol=1e-4)
    op.close()


def test_power_iteration_on_gpu_matches_oracle_estimate(dev, sol, c1_problem):
    """The library starts the power iteration from SplitMix64/Box-Muller normals of the given seed
    (the same stream synth.Stream produces), rounded to FP32; the oracle runs from that start."""
    g, s, _, f = c1_problem
    x0 = synth.Stream(11).normal(g.n).astype(np.float32).astype(np.float64).reshape(g.shape)
    L_ref = sol.power_iteration(g, s, iters=30, x0=x0)
    op = op_for(g, s)
    ft = torch.tensor(f, dtype=torch.float32, device=dev).reshape(op.data_shape)
    _, rep = op.bregman_solve(ft, 1e-3, outer=1, inner=1, prox_iters=1, L=0.0, power_iters=30, seed=11)
    assert rep["L"] == pytest.approx(L_ref, rel=1e-5)


def test_c2_bregman_residual_decreases(dev):
    """Full 64x128x128, T = 400 workload: the Bregman data residual is non-increasing (Sec. 4.6)
    and the reconstruction is non-negative."""
    w = presets.workload("c2")
    g, s = w.grid, w.sampling
    op = op_for(g, s)
    p0 = torch.tensor(w.p0(), dtype=torch.float32, device=dev).reshape(op.image_shape)
    f = op.forward(p0)
    f = f + 0.01 * float(f.abs().max()) * torch.randn_like(f)
    p, rep = op.bregman_solve(f, 2e-4, outer=3, inner=6, prox_iters=30, power_iters=10)
    r = np.array(rep["residuals"])
    assert len(r) == 3 and np.all(np.diff(r) <= 1e-6 * r[0]), r
    assert float(p.min()) >= 0.0
    err = float((p - p0).norm() / p0.norm())
    assert err < 1.0


def test_bregman_solve_checkpoint_and_resume(dev, c1_problem):
    """A solve of 4 Bregman steps equals 2 steps, a checkpoint (the image and the Bregman variable
    b_out), then 2 more steps resumed from it (warm = the image, b_in = b): bit for bit, since the
    resumed solve runs the same operations on the same data."""
    g, s, _, f = c1_problem
    op = op_for(g, s)
    ft = torch.tensor(f, dtype=torch.float32, device=dev).reshape(op.data_shape)
    _, rep = op.bregman_solve(ft, 1e-3, outer=1, inner=1, prox_iters=1, power_iters=10)
    kw = dict(inner=5, prox_iters=20, L=rep["L"])
    p4, r4 = op.bregman_solve(ft, 1e-3, outer=4, **kw)
    b = torch.full(op.data_shape, float("nan"), dtype=torch.float64, device=dev)
    p2, _ = op.bregman_solve(ft, 1e-3, outer=2, b_out=b, **kw)
    assert bool(torch.isfinite(b).all())
    p22, r22 = op.bregman_solve(ft, 1e-3, outer=2, warm=p2.clone(), b_in=b, **kw)
    assert torch.equal(p22, p4)
    assert r22["residuals"] == r4["residuals"][2:]
    op.close()

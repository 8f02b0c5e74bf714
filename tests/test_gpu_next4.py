"""Variants at the edges of the method: BPppTV+ (Sec. 6.1), regular-grid single-point sampling gSP
(Sec. 5.3, Fig. UniVsGrid) and the TV-Bregman solve on the largest workload's grid (128x256x256).

BPppTV+ is the back-projection (Eq. BP) denoised by Eq. TV+Denoise; the GPU's result is compared with
the oracle's adjoint followed by the oracle's prox at the same iteration count.  Its input carries the
adjoint's FP32 error (<= 1e-5) and the prox adds its own (<= 1e-5), so it is held to 2e-5.
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


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("name,T,alpha", [("c1", 64, 2e-3), ("c2", 16, 5e-4)])
def test_bp_tv_matches_oracle(dev, oracle_mod, name, T, alpha):
    from oracle import solver
    from paper_1605_00133_gb300.operators import PatOperator
    w = presets.shrink(presets.workload(name), T)
    g, s = w.grid, w.sampling
    f = synth.add_relative_noise(oracle_mod.forward(g, s, w.p0()), 0.01, 4)
    bp = oracle_mod.adjoint(g, s, f)
    ref = solver.tv_prox(bp, alpha, 60)
    op = PatOperator(g, s)
    got = op.bp_tv(torch.tensor(f, dtype=torch.float32, device=dev).reshape(op.data_shape), alpha, 60)
    got = got.double().cpu().numpy().reshape(g.shape)
    assert got.min() >= 0
    assert rel(got, ref) < 2e-5
    # alpha = 0: the clipped back-projection itself
    got0 = op.bp_tv(torch.tensor(f, dtype=torch.float32, device=dev).reshape(op.data_shape), 0.0, 5)
    assert rel(got0.double().cpu().numpy().reshape(g.shape), np.maximum(bp, 0)) < 1e-5
    op.close()


def test_regular_grid_sampling_matches_oracle(dev, oracle_mod):
    """gSP-16 on the 128x128 detection plane (every 4th point in y and x): the index set on the device
    is the regular grid, bit for bit, and forward and adjoint match the oracle (T = 16)."""
    from paper_1605_00133_gb300.operators import PatOperator
    w = presets.shrink(presets.workload("c2gsp"), 16)
    g, s = w.grid, w.sampling
    op = PatOperator(g, s)
    idx, _ = op.indices()
    ys, xs = np.divmod(idx, g.nx)
    assert len(idx) == 1024 and np.all(ys % 4 == 0) and np.all(xs % 4 == 0) and len(set(idx)) == 1024
    p0 = w.p0()
    x = torch.tensor(p0, dtype=torch.float32, device=dev).reshape(op.image_shape)
    assert rel(op.forward(x).double().cpu().numpy().reshape(g.T, s.m), oracle_mod.forward(g, s, p0)) < 1e-5
    y = np.random.default_rng(5).standard_normal((g.T, s.m))
    back = op.adjoint(torch.tensor(y, dtype=torch.float32, device=dev).reshape(op.data_shape))
    assert rel(back.double().cpu().numpy().reshape(g.shape), oracle_mod.adjoint(g, s, y)) < 1e-5
    op.close()


@pytest.mark.slow
def test_bregman_solve_on_the_largest_workload(dev):
    """128x256x256, dx 50 um, T = 800, rSP 4096 of 65536, 60-tube phantom: 3 Bregman steps x 4 FISTA
    iterations with the FP64 residual, objective and norm reductions.  The data residual is
    non-increasing (Sec. 4.6), the image non-negative, and each Bregman step brings the image closer
    to the phantom.  (Solves on different grids are different problems, so the FP64 oracle checks this
    grid's operator on the 2x coarser grid and the solver iterate for iterate on the 64x128x128 grid.)"""
    from paper_1605_00133_gb300.operators import PatOperator
    w = presets.workload("c4")
    g, s = w.grid, w.sampling
    op = PatOperator(g, s)
    p0 = torch.tensor(w.p0(), dtype=torch.float32, device=dev).reshape(op.image_shape)
    f = op.forward(p0)
    f = f + 0.01 * float(f.abs().max()) * torch.randn(f.shape, device=dev,
                                                      generator=torch.Generator(device=dev).manual_seed(3))
    errs = []
    for outer in (1, 2, 3):
        p, rep = op.bregman_solve(f, 2e-4, outer=outer, inner=4, prox_iters=20, power_iters=5)
        errs.append(float((p - p0).norm() / p0.norm()))
    r = np.array(rep["residuals"])
    assert len(r) == 3 and np.all(np.diff(r) <= 1e-6 * r[0]), r
    assert float(p.min()) >= 0.0
    assert errs[2] < errs[1] < errs[0] < 1.0, errs
    op.close()

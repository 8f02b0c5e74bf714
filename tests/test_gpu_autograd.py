"""Autograd wrapper: backward is the adjoint kernel; checked by central finite differences (exact for a
quadratic loss up to rounding) and against the FP64 oracle's adjoint."""
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


def _check_misfit_gradient(dev, oracle_mod, g, s, p0):
    """L(p0) = 1/2 ||C A p0 - f||^2: autograd gives A^T C^T (C A p0 - f); compared with the FP64
    oracle's adjoint of the FP64 residual, and with a central difference along a random direction
    (exact for a quadratic: (L(p+ev) - L(p-ev)) / 2e = <grad L(p), v>)."""
    from paper_1605_00133_gb300.autograd import pat_forward
    from paper_1605_00133_gb300.operators import PatOperator
    op = PatOperator(g, s)
    rng = np.random.default_rng(3)
    f = oracle_mod.forward(g, s, p0)
    f = f + 0.05 * np.abs(f).max() * rng.standard_normal((g.T, s.m))
    x = torch.tensor(p0, dtype=torch.float32, device=dev).reshape(op.image_shape).requires_grad_(True)
    ft = torch.tensor(f, dtype=torch.float32, device=dev).reshape(op.data_shape)
    r = pat_forward(x, op) - ft
    r.retain_grad()
    loss = 0.5 * (r ** 2).sum()
    loss.backward()
    grad = x.grad.double().cpu().numpy().reshape(g.shape)
    # the backward must be A^T C^T of exactly the residual the forward pass produced (for 0/1 patterns
    # the FP32 residual differs from the FP64 one by cancellation against the plane sum)
    r_used = r.grad.double().cpu().numpy().reshape(f.shape)
    ref = oracle_mod.adjoint(g, s, r_used)
    assert np.linalg.norm(grad - ref) / np.linalg.norm(ref) < 1e-5
    v = rng.standard_normal(g.shape)
    eps = 0.1 * np.linalg.norm(p0) / np.linalg.norm(v)

    def L(p):
        Ap = op.forward(torch.tensor(p, dtype=torch.float32, device=dev).reshape(op.image_shape))
        r = Ap.double().cpu().numpy().reshape(f.shape) - f
        return 0.5 * np.sum(r * r)
    fd = (L(p0 + eps * v) - L(p0 - eps * v)) / (2 * eps)
    # central differences are exact for a quadratic; what remains is FP32 rounding of C A p
    assert fd == pytest.approx(float(np.sum(grad * v)), rel=1e-3)
    op.close()


@pytest.mark.parametrize("kind", [presets.KIND_RSP, presets.KIND_SHD01])
def test_gradient_of_data_misfit(dev, oracle_mod, kind):
    g = presets.Grid(16, 32, 32, T=20, pml_size=4)
    s = presets.make_sampling(g, kind, 128, 2)
    _check_misfit_gradient(dev, oracle_mod, g, s, synth.gaussian_balls(g.shape, 2, 2.0, 5, pml=4))


def test_gradient_on_the_patterned_interrogation_workload(dev, oracle_mod):
    """The patterned-interrogation workload's grid, phantom and patterns (64x128x128, m = 2048 of
    the 16384 scrambled Hadamard 0/1 patterns of the 128x128 plane), T = 16."""
    w = presets.shrink(presets.workload("c3"), 16)
    _check_misfit_gradient(dev, oracle_mod, w.grid, w.sampling, w.p0())


def test_adjoint_function_backward_is_forward(dev, oracle_mod):
    from paper_1605_00133_gb300.autograd import pat_adjoint
    from paper_1605_00133_gb300.operators import PatOperator
    g = presets.Grid(16, 16, 16, T=12, pml_size=2)
    s = presets.make_sampling(g, presets.KIND_RSP, 60, 1)
    op = PatOperator(g, s)
    y = torch.randn(op.data_shape, device=dev, requires_grad=True)
    w = torch.randn(op.image_shape, device=dev)
    (pat_adjoint(y, op) * w).sum().backward()
    ref = oracle_mod.forward(g, s, w.double().cpu().numpy().reshape(g.shape))
    got = y.grad.double().cpu().numpy().reshape(ref.shape)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5

"""Learned warm start pipeline on a small grid: training pairs from the operators and the plain
solver, training that lowers the loss, and the warm-vs-plain evaluation, whose plain arm at the
full schedule reproduces its own reference exactly (the solver is deterministic)."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda", 0)


def test_pipeline_trains_and_evaluates(dev):
    from paper_1605_00133_gb300 import presets, unet, warmstart
    from paper_1605_00133_gb300.operators import PatOperator
    g = presets.Grid(16, 32, 32, T=24, pml_size=4)
    s = presets.make_sampling(g, presets.KIND_RSP, 256, 3)
    wl = presets.Workload("small", g, s, "tubes6", 0, bregman_outer=2, inner=10)
    op = PatOperator(g, s)
    lam = 2e-4
    _, rep = op.bregman_solve(torch.zeros(op.data_shape, device=dev), lam, outer=1, inner=1, prox_iters=1,
                              power_iters=10)
    L = rep["L"]
    pairs = warmstart.make_pairs(op, wl, 4, 100, lam, wl.bregman_outer, wl.inner, L, prox_iters=20)
    test = warmstart.make_pairs(op, wl, 1, 900, lam, wl.bregman_outer, wl.inner, L, prox_iters=20)
    net = unet.WarmStartUNet(g.nz, g.ny, g.nx, seed=0)
    net.s_in = warmstart.input_scale(pairs)
    hist = warmstart.train(net, pairs, 8, lr=1e-3, seed=0)
    assert hist[-1] < hist[0], hist
    ev = warmstart.evaluate(op, net, test, lam, wl.bregman_outer, [5, wl.inner], L, prox_iters=20)
    assert len(ev) == 1
    e = ev[0]
    assert e["plain"][-1]["rel_err"] <= 1e-6  # same schedule, same start, same L: the reference itself
    assert e["plain_seconds_to_tol"] is not None
    assert e["warm"][0]["inner"] == 0 and e["warm"][0]["rel_err"] == e["network_rel_err"]
    assert all(t["seconds"] > 0 for t in e["plain"] + e["warm"])
    op.close()

"""Learned warm start on a small grid: training pairs from the operators and the plain solver,
training that lowers the loss, and what the trained network gains.  On held-out phantoms, a solve
started from the network's output is closer to the converged plain reconstruction than the plain
cold-start solve after the same number of FISTA iterations, and reaches 10 % of it sooner."""
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


def test_trained_warm_start_beats_the_cold_start(dev):
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
    pairs = warmstart.make_pairs(op, wl, 24, 100, lam, wl.bregman_outer, 60, L, prox_iters=20)
    test = warmstart.make_pairs(op, wl, 2, 900, lam, wl.bregman_outer, 60, L, prox_iters=20)
    net = unet.WarmStartUNet(g.nz, g.ny, g.nx, seed=0)
    net.s_in = warmstart.input_scale(pairs)
    hist = warmstart.train(net, pairs, 16, lr=1e-3, seed=0)
    assert hist[-1] < 0.5 * hist[0], hist
    # the second tolerance is out of reach, so both arms run the whole schedule
    ev = warmstart.evaluate(op, net, test, lam, wl.bregman_outer, [5, 10, 20, 40], L, inner_ref=300,
                            tols=(0.10, 1e-4), prox_iters=20)
    for e in ev:
        plain = {t["inner"]: t["rel_err"] for t in e["plain"]}
        warm = {t["inner"]: t["rel_err"] for t in e["warm"]}
        print("plain", plain, "warm", warm)
        assert warm[0] == e["network_rel_err"] and e["network_rel_err"] < 1.0
        # at every budget the warm-started solve is closer to the converged reconstruction
        for n in (5, 10, 20, 40):
            assert warm[n] < plain[n], (n, warm, plain)
        # and it gets as close as the cold start's longest solve in less wall time
        t_plain = next(t["seconds"] for t in e["plain"] if t["inner"] == 40)
        t_warm = next(t["seconds"] for t in e["warm"] if t["rel_err"] <= plain[40])
        assert t_warm < t_plain, (t_warm, t_plain)
    op.close()

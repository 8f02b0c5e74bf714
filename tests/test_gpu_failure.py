"""The bounded-wait failure path of the time-step kernels, exercised without faulting the GPU.

pat_debug_copy_fault makes the line passes leave out the bulk copy of one state tile, so its
mbarrier phase never completes while nothing is in flight; each wait gives up after a few polls,
records the copy in the grid's status word and does not use the tile.  pat_device_status must then
report PAT_ERR_TIMEOUT, name the copy and clear the word, and the context must stay usable: with the
hook off, the next calls match the FP64 oracle again.  The solver reads the word itself.
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


@pytest.mark.parametrize("mask,what", [(2, b"state-1 tile"), (4, b"state-2 tile")])
def test_a_copy_that_never_lands_is_reported_and_the_context_survives(dev, oracle_mod, mask, what):
    from paper_1605_00133_gb300 import _lib
    from paper_1605_00133_gb300.operators import PatOperator
    lib = _lib.load()
    g = presets.Grid(16, 32, 32, T=8, pml_size=3)
    s = presets.make_sampling(g, presets.KIND_RSP, 200, 5)
    p0 = synth.gaussian_balls(g.shape, 2, 2.0, 7, pml=3)
    op = PatOperator(g, s)
    x = torch.tensor(p0, dtype=torch.float32, device=dev).reshape(op.image_shape)
    op.device_status(dev)  # clean start
    assert lib.pat_debug_copy_fault(op._h, mask, 4) == 0
    op.forward(x)
    with pytest.raises(_lib.PatError) as e:
        op.device_status(dev)
    assert e.value.status == 4 and what.decode() in str(e.value)
    op.device_status(dev)  # the record was cleared
    # the solver checks the word before it returns
    f = op.forward(x)
    with pytest.raises(_lib.PatError) as e:
        op.bregman_solve(f, 1e-3, outer=1, inner=2, prox_iters=5, L=1.0)
    assert e.value.status == 4
    # hook off: the same grid computes correct results again
    assert lib.pat_debug_copy_fault(op._h, 0, 0) == 0
    got = op.forward(x).double().cpu().numpy().reshape(g.T, s.m)
    assert rel(got, oracle_mod.forward(g, s, p0)) < 1e-5
    y = np.random.default_rng(3).standard_normal((g.T, s.m))
    back = op.adjoint(torch.tensor(y, dtype=torch.float32, device=dev).reshape(op.data_shape))
    assert rel(back.double().cpu().numpy().reshape(g.shape), oracle_mod.adjoint(g, s, y)) < 1e-5
    op.device_status(dev)
    op.close()


def test_tensor_core_convolution_gives_up_cleanly(dev):
    """pat_unet_debug_copy_fault makes the tcgen05 convolution issue only its first three K steps: the
    MMA thread's bounded wait for the fourth gives up, the CTA frees its tensor memory and exits, and
    pat_unet_device_status reports PAT_ERR_TIMEOUT once.  With the hook off the same convolutions
    (and a large one over many tiles, which needs tensor memory on every SM) give the results of
    before, bit for bit."""
    from paper_1605_00133_gb300 import _lib
    lib = _lib.load()
    st = torch.cuda.current_stream(dev).cuda_stream
    g = torch.Generator(device=dev).manual_seed(0)

    def conv(D, H, W, cin, cout):
        x = torch.randn((D * H * W, cin), device=dev, generator=g).to(torch.bfloat16)
        w = (0.1 * torch.randn((27, cout, cin), device=dev, generator=g)).to(torch.bfloat16)
        y = torch.zeros((D * H * W, cout), dtype=torch.bfloat16, device=dev)
        return x, w, y

    small = conv(8, 8, 8, 32, 32)
    large = conv(32, 64, 64, 16, 16)
    ref = []
    for x, w, y in (small, large):
        _lib.check(lib.pat_unet_conv3(x.data_ptr(), x.shape[1], x.shape[1], w.data_ptr(), y.shape[1],
                                      y.data_ptr(), y.shape[1], *((8, 8, 8) if x is small[0] else (32, 64, 64)),
                                      0, st))
        ref.append(y.clone())
    _lib.check(lib.pat_unet_device_status(st))
    x, w, y = small
    try:
        _lib.check(lib.pat_unet_debug_copy_fault(3, 4))
        _lib.check(lib.pat_unet_conv3(x.data_ptr(), 32, 32, w.data_ptr(), 32, y.data_ptr(), 32, 8, 8, 8, 0, st))
        with pytest.raises(_lib.PatError) as e:
            _lib.check(lib.pat_unet_device_status(st))
        assert e.value.status == 4
    finally:
        _lib.check(lib.pat_unet_debug_copy_fault(-1, 0))
    _lib.check(lib.pat_unet_device_status(st))  # cleared
    for (x, w, y), r, dims in ((small, ref[0], (8, 8, 8)), (large, ref[1], (32, 64, 64))):
        y.zero_()
        _lib.check(lib.pat_unet_conv3(x.data_ptr(), x.shape[1], x.shape[1], w.data_ptr(), y.shape[1],
                                      y.data_ptr(), y.shape[1], *dims, 0, st))
        torch.cuda.synchronize()
        assert torch.equal(y, r)
    _lib.check(lib.pat_unet_device_status(st))

"""pat_forward_noalloc: the forward operator for callers that cannot allocate device memory at call
time (reconstruction loops that reserve their whole device budget at start-up).  Its scratch is a
static 64 MiB device array inside libpat, so its results must equal pat_forward's and the FP64
oracle's, call after call, and grids that do not fit must be refused with a clear message.

This file is named to be collected last, so a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1605_00133_gb300 import presets  # noqa: E402

TOL = 1e-5  # the parity tolerance of the FP32 operators


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda", 0)


def _call(lib, fn, op, x, out):
    stream = torch.cuda.current_stream(x.device).cuda_stream
    st = getattr(lib, fn)(op._h, x.data_ptr(), out.data_ptr(), stream)
    if st != 0:
        raise RuntimeError(f"{fn}: {st} {lib.pat_last_error().decode()}")


@pytest.mark.parametrize("kind", [presets.KIND_RSP, presets.KIND_FULL])
def test_noalloc_forward_matches_pat_forward_twice(dev, kind):
    from paper_1605_00133_gb300 import _lib
    from paper_1605_00133_gb300.operators import PatOperator
    lib = _lib.load()
    w = presets.workload("c1")
    g = w.grid
    s = presets.make_sampling(g, kind, 256, 3)
    op = PatOperator(g, s)
    rng = np.random.default_rng(21)
    for call in range(2):  # the array keeps the previous call's contents: results must not depend on it
        p0 = torch.tensor(w.p0(seed_offset=call) + 0.1 * rng.standard_normal(g.shape),
                          dtype=torch.float32, device=dev).reshape(op.image_shape)
        ref = torch.empty(op.data_shape, device=dev)
        got = torch.full(op.data_shape, float("nan"), device=dev)
        _call(lib, "pat_forward", op, p0, ref)
        _call(lib, "pat_forward_noalloc", op, p0, got)
        torch.cuda.synchronize()
        a, b = got.double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= TOL, call
    op.close()


def test_noalloc_forward_matches_the_oracle(oracle_mod, dev):
    """Against the FP64 oracle directly (not only against pat_forward, which shares its kernels):
    the c1 workload, two calls in a row with different phantoms."""
    from paper_1605_00133_gb300 import _lib
    from paper_1605_00133_gb300.operators import PatOperator
    lib = _lib.load()
    w = presets.workload("c1")
    g, s = w.grid, w.sampling
    op = PatOperator(g, s)
    for call in range(2):
        p0 = w.p0(seed_offset=call)
        x = torch.tensor(p0, dtype=torch.float32, device=dev).reshape(op.image_shape)
        got = torch.full(op.data_shape, float("nan"), device=dev)
        _call(lib, "pat_forward_noalloc", op, x, got)
        torch.cuda.synchronize()
        ref = oracle_mod.forward(g, s, p0)
        a = got.double().cpu().numpy().reshape(ref.shape)
        assert np.linalg.norm(a - ref) / np.linalg.norm(ref) <= TOL, call
    op.close()


def test_noalloc_forward_on_the_c2_grid(dev):
    """64x128x128, T = 400, point sampling: the largest workload the 64 MiB array is sized for."""
    from paper_1605_00133_gb300 import _lib
    from paper_1605_00133_gb300.operators import PatOperator
    lib = _lib.load()
    w = presets.workload("c2")
    op = PatOperator(w.grid, w.sampling)
    p0 = torch.tensor(w.p0(), dtype=torch.float32, device=dev).reshape(op.image_shape)
    ref = torch.empty(op.data_shape, device=dev)
    got = torch.empty(op.data_shape, device=dev)
    _call(lib, "pat_forward", op, p0, ref)
    _call(lib, "pat_forward_noalloc", op, p0, got)
    torch.cuda.synchronize()
    a, b = got.double().cpu().numpy(), ref.double().cpu().numpy()
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= TOL
    op.close()


def test_noalloc_rejects_grids_beyond_the_array(dev):
    from paper_1605_00133_gb300 import _lib
    from paper_1605_00133_gb300.operators import PatOperator
    lib = _lib.load()
    w = presets.workload("c2")
    g = w.grid
    g2 = presets.Grid(g.nz, g.ny, g.nx, dx=g.dx, T=g.T, pml_size=g.pml_size, batch=2)
    op = PatOperator(g2, w.sampling)
    p0 = torch.zeros(op.image_shape, device=dev)
    f = torch.zeros(op.data_shape, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    st = lib.pat_forward_noalloc(op._h, ctypes.c_void_p(p0.data_ptr()), ctypes.c_void_p(f.data_ptr()),
                                 ctypes.c_void_p(stream))
    assert st == 1
    assert b"static scratch holds" in lib.pat_last_error()
    op.close()

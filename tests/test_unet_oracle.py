"""Pins of the FP64 U-Net reference (oracle/unet.py) against things other than itself: the
convolution against its defining sum written as loops, pooling/upsampling identities, and every
parameter gradient against central finite differences of the loss."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet as ou  # noqa: E402


def test_conv3_matches_the_defining_sum():
    rng = np.random.default_rng(0)
    cin, cout, D, H, W = 2, 3, 4, 3, 5
    x = rng.standard_normal((cin, D, H, W))
    w = rng.standard_normal((27, cout, cin))
    y = ou.conv3(torch.tensor(x), torch.tensor(w)).numpy()
    ref = np.zeros((cout, D, H, W))
    for co in range(cout):
        for z in range(D):
            for yy in range(H):
                for xx in range(W):
                    s = 0.0
                    for t in range(27):
                        dz, dy, dx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
                        zz, y2, x2 = z + dz, yy + dy, xx + dx
                        if 0 <= zz < D and 0 <= y2 < H and 0 <= x2 < W:
                            s += sum(w[t, co, ci] * x[ci, zz, y2, x2] for ci in range(cin))
                    ref[co, z, yy, xx] = s
    assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()


def test_pool_of_upsampled_is_identity_and_pool_averages():
    x = torch.randn(3, 2, 4, 2, dtype=torch.float64)
    assert torch.allclose(ou.pool(ou.up(x)), x, atol=1e-15)
    v = torch.arange(8, dtype=torch.float64).reshape(1, 2, 2, 2)
    assert float(ou.pool(v)[0, 0, 0, 0]) == 3.5


def test_gradients_match_central_differences():
    import paper_1605_00133_gb300.unet as un  # parameter initialisation only (no device code)
    g = torch.Generator().manual_seed(1)
    params = un.init_params(3)
    xin = torch.rand((8, 8, 8), generator=g, dtype=torch.float64)
    target = torch.rand((8, 8, 8), generator=g, dtype=torch.float64)
    loss, _, grads = ou.loss_and_grads(params, xin, target, 1.0)
    p64 = {k: v.double() for k, v in params.items()}
    rng = np.random.default_rng(2)
    for name in ("e1a", "e4b", "d3a", "d1b", "head"):
        flat = p64[name].reshape(-1)
        for _ in range(2):
            i = int(rng.integers(flat.numel()))
            eps = 1e-5 * max(1.0, abs(float(flat[i])))

            def L(delta):
                q = {k: v.clone() for k, v in p64.items()}
                q[name].reshape(-1)[i] += delta
                out = ou.forward(q, xin, 1.0)
                return float(((out - target) ** 2).mean())
            fd = (L(eps) - L(-eps)) / (2 * eps)
            an = float(grads[name].reshape(-1)[i])
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-8) + 1e-10, (name, i, fd, an)

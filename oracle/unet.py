"""FP64 CPU reference of the learned warm start's 3D U-Net (forward, loss and every gradient).

TEST INFRASTRUCTURE ONLY: the test-suite and the benchmark are the only users; the library never
imports this module.  The paper has no learned component (the network warm-starts the TV-Bregman
solver of Sec. 4.5-4.6 / App. B), so this module restates the network's definition with plain
PyTorch CPU operations in double precision, and torch.autograd supplies the gradients:
  conv3       3x3x3 convolution, stride 1, zero padding 1, no bias; weights [27][Cout][Cin] with
              tap t = 9 (dz+1) + 3 (dy+1) + (dx+1), i.e. y[co](z,y,x) = sum_t sum_ci
              w[t][co][ci] x[ci](z+dz, y+dy, x+dx)
  pool        2x2x2 average;  up  nearest-neighbour x2;  cat  [upsampled | skip] along channels
  head        out = head[16] + sum_c head[c] h[c]
  loss        mean over voxels of (out - target)^2
Volumes are [C][D][H][W] here (the GPU stores them channels-last).  Pins: tests/test_unet_oracle.py
(the convolution against its defining sum written as loops on tiny inputs, and the gradients
against central finite differences).
"""
from __future__ import annotations

import torch
import torch.nn.functional as F


def conv3(x: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    """x [Cin][D][H][W], w [27][Cout][Cin] -> [Cout][D][H][W]."""
    cout, cin = w.shape[1], w.shape[2]
    k = w.reshape(3, 3, 3, cout, cin).permute(3, 4, 0, 1, 2)  # [Cout][Cin][dz][dy][dx]
    return F.conv3d(x.unsqueeze(0), k, padding=1)[0]


def pool(x):
    return F.avg_pool3d(x.unsqueeze(0), 2)[0]


def up(x):
    return x.repeat_interleave(2, 1).repeat_interleave(2, 2).repeat_interleave(2, 3)


def forward(params: dict, xin: torch.Tensor, s_in: float) -> torch.Tensor:
    """params: tensors laid out as the library's unet.init_params returns them; xin [D][H][W];
    returns out [D][H][W]."""
    w = {k: v.double() for k, v in params.items()}
    D, H, W = xin.shape
    x = torch.zeros((16, D, H, W), dtype=torch.float64)
    x[0] = s_in * xin.double()
    r = torch.relu
    t1 = r(conv3(x, w["e1a"]))
    s1 = r(conv3(t1, w["e1b"]))
    t2 = r(conv3(pool(s1), w["e2a"]))
    s2 = r(conv3(t2, w["e2b"]))
    t3 = r(conv3(pool(s2), w["e3a"]))
    s3 = r(conv3(t3, w["e3b"]))
    t4 = r(conv3(pool(s3), w["e4a"]))
    u4 = r(conv3(t4, w["e4b"]))
    u3 = r(conv3(r(conv3(torch.cat([up(u4), s3]), w["d3a"])), w["d3b"]))
    u2 = r(conv3(r(conv3(torch.cat([up(u3), s2]), w["d2a"])), w["d2b"]))
    h = r(conv3(r(conv3(torch.cat([up(u2), s1]), w["d1a"])), w["d1b"]))
    hd = w["head"]
    return hd[16] + torch.einsum("c,cdhw->dhw", hd[:16], h)


def loss_and_grads(params: dict, xin, target, s_in: float):
    """(loss, out, {name: dloss/dparam}) in FP64."""
    p = {k: v.detach().double().clone().requires_grad_(True) for k, v in params.items()}
    out = forward(p, xin, s_in)
    loss = ((out - target.double()) ** 2).mean()
    loss.backward()
    return float(loss.detach()), out.detach(), {k: v.grad.detach() for k, v in p.items()}

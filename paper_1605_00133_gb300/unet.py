"""Learned warm start for the TV-Bregman solver: a 3D U-Net that maps the back-projection A^T C^T f
to a starting image (the paper has no learned component; the solver it warm-starts is Sec. 4.5-4.6
and App. B, and stays the fallback and the reference the warm start's error is measured against).

Architecture: 4 levels with 16/32/64/128 channels, two 3x3x3 convolutions + ReLU per level and
side, 2x2x2 average pooling down, nearest-neighbour upsampling and channel concatenation
[upsampled | skip] on the way up, and a 1x1x1 output layer with bias.  Every layer runs in libpat's
kernels (include/pat_unet.h): BF16 activations and weights on the tensor cores with FP32
accumulation, FP32 master weights and Adam moments.  PyTorch only provides device memory and the
stream.

Training pairs are (A^T C^T f, TV-Bregman reconstruction of f) for seeded vessel phantoms; the loss
is the mean squared error.
"""
from __future__ import annotations

import torch

from . import _lib

# name: (input channels, output channels, level)
LAYERS = {
    "e1a": (16, 16, 0), "e1b": (16, 16, 0),
    "e2a": (16, 32, 1), "e2b": (32, 32, 1),
    "e3a": (32, 64, 2), "e3b": (64, 64, 2),
    "e4a": (64, 128, 3), "e4b": (128, 128, 3),
    "d3a": (192, 64, 2), "d3b": (64, 64, 2),
    "d2a": (96, 32, 1), "d2b": (32, 32, 1),
    "d1a": (48, 16, 0), "d1b": (16, 16, 0),
}


def init_params(seed: int = 0) -> dict:
    """He-normal FP32 weights [27][cout][cin] per layer and the output layer (16 weights + bias)."""
    g = torch.Generator().manual_seed(seed)
    p = {}
    for name, (cin, cout, _) in LAYERS.items():
        std = (2.0 / (27 * cin)) ** 0.5
        p[name] = torch.randn((27, cout, cin), generator=g, dtype=torch.float32) * std
    p["head"] = torch.cat([torch.randn(16, generator=g) * (1.0 / 16) ** 0.5, torch.zeros(1)]).float()
    return p


class WarmStartUNet:
    """The network on one GPU for volumes D x H x W (each divisible by 8), one sample at a time."""

    def __init__(self, D: int, H: int, W: int, device=None, seed: int = 0, params: dict = None):
        if D % 8 or H % 8 or W % 8:
            raise ValueError("U-Net volume sides must be divisible by 8")
        self.L = _lib.load()
        self.dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.dims = [(D >> k, H >> k, W >> k) for k in range(4)]
        self.V = [d * h * w for d, h, w in self.dims]
        params = init_params(seed) if params is None else params
        # one flat FP32 parameter vector (conv weights in LAYERS order, then the head), its gradient
        # and the Adam moments
        sizes = [27 * c[0] * c[1] for c in LAYERS.values()] + [17]
        self.n_params = sum(sizes)
        self.P = torch.zeros(self.n_params, dtype=torch.float32, device=self.dev)
        self.G = torch.zeros_like(self.P)
        self.M1 = torch.zeros_like(self.P)
        self.M2 = torch.zeros_like(self.P)
        self.off = {}
        o = 0
        for name, n in zip(list(LAYERS) + ["head"], sizes):
            self.off[name] = (o, n)
            self.P[o:o + n] = params[name].reshape(-1).to(self.dev)
            o += n
        self.wb = {n: torch.empty((27, c[1], c[0]), dtype=torch.bfloat16, device=self.dev) for n, c in LAYERS.items()}
        self.wt = {n: torch.empty((27, c[0], c[1]), dtype=torch.bfloat16, device=self.dev) for n, c in LAYERS.items()}
        self.step_count = 0
        V0, V1, V2, V3 = self.V

        def a(v, c):
            return torch.zeros((v, c), dtype=torch.bfloat16, device=self.dev)

        # activations (channels-last BF16); concatenations are [upsampled | skip]
        self.x16, self.t1, self.c1 = a(V0, 16), a(V0, 16), a(V0, 48)
        self.p1, self.t2, self.c2 = a(V1, 16), a(V1, 32), a(V1, 96)
        self.p2, self.t3, self.c3 = a(V2, 32), a(V2, 64), a(V2, 192)
        self.p3, self.t4, self.u4 = a(V3, 64), a(V3, 128), a(V3, 128)
        self.t3b, self.u3 = a(V2, 64), a(V2, 64)
        self.t2b, self.u2 = a(V1, 32), a(V1, 32)
        self.t1b, self.h = a(V0, 16), a(V0, 16)
        self.out = torch.zeros(V0, dtype=torch.float32, device=self.dev)
        # gradients
        self.dh, self.dt1b, self.dc1 = a(V0, 16), a(V0, 16), a(V0, 48)
        self.du2, self.dt2b, self.dc2 = a(V1, 32), a(V1, 32), a(V1, 96)
        self.du3, self.dt3b, self.dc3 = a(V2, 64), a(V2, 64), a(V2, 192)
        self.du4, self.dt4, self.dp3 = a(V3, 128), a(V3, 128), a(V3, 64)
        self.dt3, self.dp2, self.dt2, self.dp1, self.dt1 = a(V2, 64), a(V2, 32), a(V1, 32), a(V1, 16), a(V0, 16)
        ws = max(self.L.pat_unet_wgrad_scratch(c[0], c[1], *self.dims[c[2]]) for c in LAYERS.values())
        self.wscratch = torch.empty(ws, dtype=torch.float32, device=self.dev)
        self.hscratch = torch.empty(self.L.pat_unet_head_scratch(V0), dtype=torch.float64, device=self.dev)
        self.loss_buf = torch.zeros(1, dtype=torch.float64, device=self.dev)
        self.s_in = 1.0
        self._cast()

    # ------------------------------------------------------------------ helpers
    def _st(self):
        return torch.cuda.current_stream(self.dev).cuda_stream

    @staticmethod
    def _p(t, ch=0):
        """device address of channel `ch` of a channels-last BF16 tensor"""
        return t.data_ptr() + 2 * ch

    def _w32(self, name):
        return self.P.data_ptr() + 4 * self.off[name][0]

    def _g32(self, name):
        return self.G.data_ptr() + 4 * self.off[name][0]

    def _cast(self):
        for name, (cin, cout, _) in LAYERS.items():
            _lib.check(self.L.pat_unet_cast_weights(self._w32(name), cin, cout, self.wb[name].data_ptr(),
                                                    self.wt[name].data_ptr(), self._st()))

    def _conv(self, x, ldx, cin, w, cout, y, ldy, lev, relu):
        D, H, W = self.dims[lev]
        _lib.check(self.L.pat_unet_conv3(x, ldx, cin, w, cout, y, ldy, D, H, W, int(relu), self._st()))

    def _wgrad(self, name, x, ldx, dy, ldy):
        cin, cout, lev = LAYERS[name]
        D, H, W = self.dims[lev]
        _lib.check(self.L.pat_unet_conv3_wgrad(x, ldx, cin, dy, ldy, cout, D, H, W, self.wscratch.data_ptr(),
                                               self._g32(name), self._st()))

    def _relu_bwd(self, g, ldg, y, ldy, C, lev):
        _lib.check(self.L.pat_unet_relu_bwd(g, ldg, y, ldy, C, self.V[lev], self._st()))

    # ------------------------------------------------------------------ forward
    def forward(self, xin: torch.Tensor) -> torch.Tensor:
        """xin: FP32 with V elements (the back-projection); returns the FP32 output [V] (a buffer of
        the network, overwritten by the next call)."""
        L, st, p = self.L, self._st(), self._p
        d0, d1, d2, d3 = self.dims
        xin = xin.reshape(-1).contiguous()
        _lib.check(L.pat_unet_input(xin.data_ptr(), float(self.s_in), self.V[0], self.x16.data_ptr(), st))
        wb = {k: v.data_ptr() for k, v in self.wb.items()}
        self._conv(p(self.x16), 16, 16, wb["e1a"], 16, p(self.t1), 16, 0, True)
        self._conv(p(self.t1), 16, 16, wb["e1b"], 16, p(self.c1, 32), 48, 0, True)
        _lib.check(L.pat_unet_pool(p(self.c1, 32), 48, 16, *d0, p(self.p1), 16, st))
        self._conv(p(self.p1), 16, 16, wb["e2a"], 32, p(self.t2), 32, 1, True)
        self._conv(p(self.t2), 32, 32, wb["e2b"], 32, p(self.c2, 64), 96, 1, True)
        _lib.check(L.pat_unet_pool(p(self.c2, 64), 96, 32, *d1, p(self.p2), 32, st))
        self._conv(p(self.p2), 32, 32, wb["e3a"], 64, p(self.t3), 64, 2, True)
        self._conv(p(self.t3), 64, 64, wb["e3b"], 64, p(self.c3, 128), 192, 2, True)
        _lib.check(L.pat_unet_pool(p(self.c3, 128), 192, 64, *d2, p(self.p3), 64, st))
        self._conv(p(self.p3), 64, 64, wb["e4a"], 128, p(self.t4), 128, 3, True)
        self._conv(p(self.t4), 128, 128, wb["e4b"], 128, p(self.u4), 128, 3, True)
        _lib.check(L.pat_unet_up(p(self.u4), 128, 128, *d3, p(self.c3), 192, st))
        self._conv(p(self.c3), 192, 192, wb["d3a"], 64, p(self.t3b), 64, 2, True)
        self._conv(p(self.t3b), 64, 64, wb["d3b"], 64, p(self.u3), 64, 2, True)
        _lib.check(L.pat_unet_up(p(self.u3), 64, 64, *d2, p(self.c2), 96, st))
        self._conv(p(self.c2), 96, 96, wb["d2a"], 32, p(self.t2b), 32, 1, True)
        self._conv(p(self.t2b), 32, 32, wb["d2b"], 32, p(self.u2), 32, 1, True)
        _lib.check(L.pat_unet_up(p(self.u2), 32, 32, *d1, p(self.c1), 48, st))
        self._conv(p(self.c1), 48, 48, wb["d1a"], 16, p(self.t1b), 16, 0, True)
        self._conv(p(self.t1b), 16, 16, wb["d1b"], 16, p(self.h), 16, 0, True)
        _lib.check(L.pat_unet_head(p(self.h), self._w32("head"), self.V[0], self.out.data_ptr(), st))
        return self.out

    # ------------------------------------------------------------------ backward (after forward)
    def backward(self, target: torch.Tensor) -> torch.Tensor:
        """Gradient of the mean squared error against target (FP32, V elements) into self.G; returns
        the loss (FP64 device scalar)."""
        L, st, p = self.L, self._st(), self._p
        d0, d1, d2, d3 = self.dims
        wt = {k: v.data_ptr() for k, v in self.wt.items()}
        target = target.reshape(-1).contiguous()
        _lib.check(L.pat_unet_head_bwd(p(self.h), self._w32("head"), self.out.data_ptr(), target.data_ptr(),
                                       self.V[0], p(self.dh), self._g32("head"), self.loss_buf.data_ptr(),
                                       self.hscratch.data_ptr(), st))
        # level 1, decoder
        self._relu_bwd(p(self.dh), 16, p(self.h), 16, 16, 0)
        self._wgrad("d1b", p(self.t1b), 16, p(self.dh), 16)
        self._conv(p(self.dh), 16, 16, wt["d1b"], 16, p(self.dt1b), 16, 0, False)
        self._relu_bwd(p(self.dt1b), 16, p(self.t1b), 16, 16, 0)
        self._wgrad("d1a", p(self.c1), 48, p(self.dt1b), 16)
        self._conv(p(self.dt1b), 16, 16, wt["d1a"], 48, p(self.dc1), 48, 0, False)
        _lib.check(L.pat_unet_up_bwd(p(self.dc1), 48, 32, *d1, p(self.du2), 32, st))
        # level 2, decoder
        self._relu_bwd(p(self.du2), 32, p(self.u2), 32, 32, 1)
        self._wgrad("d2b", p(self.t2b), 32, p(self.du2), 32)
        self._conv(p(self.du2), 32, 32, wt["d2b"], 32, p(self.dt2b), 32, 1, False)
        self._relu_bwd(p(self.dt2b), 32, p(self.t2b), 32, 32, 1)
        self._wgrad("d2a", p(self.c2), 96, p(self.dt2b), 32)
        self._conv(p(self.dt2b), 32, 32, wt["d2a"], 96, p(self.dc2), 96, 1, False)
        _lib.check(L.pat_unet_up_bwd(p(self.dc2), 96, 64, *d2, p(self.du3), 64, st))
        # level 3, decoder
        self._relu_bwd(p(self.du3), 64, p(self.u3), 64, 64, 2)
        self._wgrad("d3b", p(self.t3b), 64, p(self.du3), 64)
        self._conv(p(self.du3), 64, 64, wt["d3b"], 64, p(self.dt3b), 64, 2, False)
        self._relu_bwd(p(self.dt3b), 64, p(self.t3b), 64, 64, 2)
        self._wgrad("d3a", p(self.c3), 192, p(self.dt3b), 64)
        self._conv(p(self.dt3b), 64, 64, wt["d3a"], 192, p(self.dc3), 192, 2, False)
        _lib.check(L.pat_unet_up_bwd(p(self.dc3), 192, 128, *d3, p(self.du4), 128, st))
        # level 4
        self._relu_bwd(p(self.du4), 128, p(self.u4), 128, 128, 3)
        self._wgrad("e4b", p(self.t4), 128, p(self.du4), 128)
        self._conv(p(self.du4), 128, 128, wt["e4b"], 128, p(self.dt4), 128, 3, False)
        self._relu_bwd(p(self.dt4), 128, p(self.t4), 128, 128, 3)
        self._wgrad("e4a", p(self.p3), 64, p(self.dt4), 128)
        self._conv(p(self.dt4), 128, 128, wt["e4a"], 64, p(self.dp3), 64, 3, False)
        # level 3, encoder (the skip's gradient from the concatenation plus the pooled path)
        _lib.check(L.pat_unet_pool_bwd_add(p(self.dp3), 64, 64, *d2, p(self.dc3, 128), 192, st))
        self._relu_bwd(p(self.dc3, 128), 192, p(self.c3, 128), 192, 64, 2)
        self._wgrad("e3b", p(self.t3), 64, p(self.dc3, 128), 192)
        self._conv(p(self.dc3, 128), 192, 64, wt["e3b"], 64, p(self.dt3), 64, 2, False)
        self._relu_bwd(p(self.dt3), 64, p(self.t3), 64, 64, 2)
        self._wgrad("e3a", p(self.p2), 32, p(self.dt3), 64)
        self._conv(p(self.dt3), 64, 64, wt["e3a"], 32, p(self.dp2), 32, 2, False)
        # level 2, encoder
        _lib.check(L.pat_unet_pool_bwd_add(p(self.dp2), 32, 32, *d1, p(self.dc2, 64), 96, st))
        self._relu_bwd(p(self.dc2, 64), 96, p(self.c2, 64), 96, 32, 1)
        self._wgrad("e2b", p(self.t2), 32, p(self.dc2, 64), 96)
        self._conv(p(self.dc2, 64), 96, 32, wt["e2b"], 32, p(self.dt2), 32, 1, False)
        self._relu_bwd(p(self.dt2), 32, p(self.t2), 32, 32, 1)
        self._wgrad("e2a", p(self.p1), 16, p(self.dt2), 32)
        self._conv(p(self.dt2), 32, 32, wt["e2a"], 16, p(self.dp1), 16, 1, False)
        # level 1, encoder
        _lib.check(L.pat_unet_pool_bwd_add(p(self.dp1), 16, 16, *d0, p(self.dc1, 32), 48, st))
        self._relu_bwd(p(self.dc1, 32), 48, p(self.c1, 32), 48, 16, 0)
        self._wgrad("e1b", p(self.t1), 16, p(self.dc1, 32), 48)
        self._conv(p(self.dc1, 32), 48, 16, wt["e1b"], 16, p(self.dt1), 16, 0, False)
        self._relu_bwd(p(self.dt1), 16, p(self.t1), 16, 16, 0)
        self._wgrad("e1a", p(self.x16), 16, p(self.dt1), 16)
        return self.loss_buf

    def adam_step(self, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8) -> None:
        self.step_count += 1
        _lib.check(self.L.pat_unet_adam(self.P.data_ptr(), self.G.data_ptr(), self.M1.data_ptr(), self.M2.data_ptr(),
                                        self.n_params, lr, b1, b2, eps, self.step_count, self._st()))
        self._cast()

    def train_step(self, xin, target, lr=1e-3) -> torch.Tensor:
        self.forward(xin)
        loss = self.backward(target)
        self.adam_step(lr)
        return loss

    def _unflat(self, vec) -> dict:
        out = {}
        for name in list(LAYERS) + ["head"]:
            o, n = self.off[name]
            v = vec[o:o + n].detach().cpu()
            out[name] = v.reshape(27, LAYERS[name][1], LAYERS[name][0]) if name in LAYERS else v
        return out

    def params(self) -> dict:
        """Current FP32 parameters, laid out as init_params returns them (on the CPU)."""
        return self._unflat(self.P)

    def grads(self) -> dict:
        """Gradient of the last backward(), same layout."""
        return self._unflat(self.G)

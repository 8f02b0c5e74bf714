"""Python face of libpat: the PAT operators A, A^T and C on one GPU (arXiv:1605.00133, Sec. 4.3).

    op = PatOperator(grid, sampling)          # pat_create_grid
    f = op.forward(p0)                        # pat_forward,  f = C A p0      (Eq. Fwd)
    p = op.adjoint(f)                         # pat_adjoint,  p = A^T C^T f   (Eq. BP)

Tensors are torch CUDA float32, contiguous; calls run on torch's current stream.  PyTorch only
provides device memory and the stream: the computation is libpat's.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from .presets import KIND_FULL, KIND_RSP, KIND_SHD01, KIND_SHDPM, Grid, Sampling


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


class PatOperator:
    def __init__(self, grid: Grid, sampling: Sampling):
        lib = _lib.load()
        if not torch.cuda.is_available():
            raise RuntimeError("PatOperator needs a CUDA device; libpat has no CPU fallback")
        self.grid = grid
        self.sampling = sampling
        self.device = torch.device("cuda", torch.cuda.current_device())
        torch.cuda.init()
        d = _lib.GridDesc(grid.nz, grid.ny, grid.nx, grid.dx, grid.c, grid.rho0, grid.cfl, grid.dt,
                          grid.T, grid.pml_size, grid.pml_alpha, grid.sensor_z, grid.batch)
        keep = []

        def iptr(a):
            if a is None:
                return None
            arr = np.ascontiguousarray(a, dtype=np.int32)
            keep.append(arr)
            return arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))

        s = _lib.SamplingDesc(sampling.kind, sampling.m, iptr(sampling.indices), iptr(sampling.perm),
                              iptr(sampling.rows))
        h = ctypes.c_void_p()
        _lib.check(lib.pat_create_grid(ctypes.byref(d), ctypes.byref(s), ctypes.byref(h)))
        self._h = h
        n_img, n_dat, m, dt = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_double()
        _lib.check(lib.pat_grid_info(h, ctypes.byref(n_img), ctypes.byref(n_dat), ctypes.byref(m),
                                     ctypes.byref(dt)))
        self.n_image, self.n_data, self.m, self.dt = n_img.value, n_dat.value, m.value, dt.value
        self.B = grid.batch

    # ------------------------------------------------------------------ shapes
    @property
    def image_shape(self):
        return (self.B, self.grid.nz, self.grid.ny, self.grid.nx)

    @property
    def data_shape(self):
        return (self.B, self.grid.T, self.m)

    @property
    def workspace_bytes(self) -> int:
        return int(_lib.load().pat_workspace_bytes(self._h))

    def _check_tensor(self, t: torch.Tensor, shape, name):
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.float32:
            raise TypeError(f"{name} must be a CUDA float32 tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() != int(np.prod(shape)):
            raise ValueError(f"{name} has {t.numel()} elements, expected shape {shape}")

    # ------------------------------------------------------------------ operators
    def forward_into(self, p0: torch.Tensor, f: torch.Tensor) -> torch.Tensor:
        self._check_tensor(p0, self.image_shape, "p0")
        self._check_tensor(f, self.data_shape, "f")
        _lib.check(_lib.load().pat_forward(self._h, p0.data_ptr(), f.data_ptr(), _stream_ptr(p0.device)))
        return f

    def adjoint_into(self, f: torch.Tensor, p: torch.Tensor) -> torch.Tensor:
        self._check_tensor(f, self.data_shape, "f")
        self._check_tensor(p, self.image_shape, "p")
        _lib.check(_lib.load().pat_adjoint(self._h, f.data_ptr(), p.data_ptr(), _stream_ptr(f.device)))
        return p

    def forward(self, p0: torch.Tensor) -> torch.Tensor:
        f = torch.empty(self.data_shape, device=p0.device, dtype=torch.float32)
        return self.forward_into(p0.contiguous(), f)

    def adjoint(self, f: torch.Tensor) -> torch.Tensor:
        p = torch.empty(self.image_shape, device=f.device, dtype=torch.float32)
        return self.adjoint_into(f.contiguous(), p)

    def sample(self, pbar: torch.Tensor) -> torch.Tensor:
        """C per time point: pbar [B][nt][Ny*Nx] -> [B][nt][m]."""
        nt = pbar.numel() // (self.B * self.grid.m_plane)
        self._check_tensor(pbar, (self.B, nt, self.grid.m_plane), "pbar")
        f = torch.empty((self.B, nt, self.m), device=pbar.device, dtype=torch.float32)
        _lib.check(_lib.load().pat_sample(self._h, pbar.data_ptr(), f.data_ptr(), nt,
                                          _stream_ptr(pbar.device)))
        return f

    def sample_adjoint(self, f: torch.Tensor) -> torch.Tensor:
        """C^T per time point: f [B][nt][m] -> [B][nt][Ny*Nx]."""
        nt = f.numel() // (self.B * self.m) if self.m else 0
        self._check_tensor(f, (self.B, nt, self.m), "f")
        pbar = torch.empty((self.B, nt, self.grid.m_plane), device=f.device, dtype=torch.float32)
        _lib.check(_lib.load().pat_sample_adjoint(self._h, f.data_ptr(), pbar.data_ptr(), nt,
                                                  _stream_ptr(f.device)))
        return pbar

    def indices(self):
        """The index sets held on the device (pat_get_indices): POINTS -> (idx, None),
        HADAMARD* -> (perm, rows), FULL -> (None, None)."""
        k = self.sampling.kind
        if k == KIND_FULL:
            return None, None
        a = np.zeros(self.m if k == KIND_RSP else self.grid.m_plane, dtype=np.int32)
        r = np.zeros(self.m, dtype=np.int32) if k in (KIND_SHD01, KIND_SHDPM) else None
        ip = ctypes.POINTER(ctypes.c_int32)
        _lib.check(_lib.load().pat_get_indices(self._h, a.ctypes.data_as(ip),
                                               r.ctypes.data_as(ip) if r is not None else None))
        return a, r

    # ------------------------------------------------------------------ variational reconstruction
    def tv_prox(self, p: torch.Tensor, alpha: float, iters: int = 200, out: torch.Tensor = None):
        """argmin_{q >= 0} 1/2 ||q - p||^2 + alpha TV(q) (pat_tv_prox, Neumann boundary)."""
        self._check_tensor(p, self.image_shape, "p")
        if out is None:
            out = torch.empty_like(p)
        self._check_tensor(out, self.image_shape, "out")
        _lib.check(_lib.load().pat_tv_prox(self._h, p.data_ptr(), out.data_ptr(), float(alpha), int(iters),
                                           0, _stream_ptr(p.device)))
        return out

    def bp_tv(self, f: torch.Tensor, alpha: float, iters: int = 200, out: torch.Tensor = None):
        """BPppTV+: argmin_{q >= 0} 1/2 ||q - A^T C^T f||^2 + alpha TV(q) (pat_bp_tv)."""
        self._check_tensor(f, self.data_shape, "f")
        if out is None:
            out = torch.empty(self.image_shape, device=f.device, dtype=torch.float32)
        self._check_tensor(out, self.image_shape, "out")
        _lib.check(_lib.load().pat_bp_tv(self._h, f.data_ptr(), out.data_ptr(), float(alpha), int(iters),
                                         _stream_ptr(f.device)))
        return out

    def bregman_solve(self, f: torch.Tensor, lam: float, outer: int = 5, inner: int = 50,
                      prox_iters: int = 100, L: float = 0.0, power_iters: int = 20, seed: int = 0,
                      step_scale: float = 1.8, max_backtrack: int = 5, stall: int = 5,
                      warm: torch.Tensor = None, out: torch.Tensor = None, b_in: torch.Tensor = None,
                      b_out: torch.Tensor = None):
        """TV+ (outer = 1) or TV+Br reconstruction from data f (pat_bregman_solve).  b_in / b_out:
        float64 device tensors of the data's shape, the Bregman variable to resume from / saved after
        the last step (with warm = the image, a checkpoint of the solve).  Returns (p, report dict)."""
        for name, b in (("b_in", b_in), ("b_out", b_out)):
            if b is not None and (b.dtype != torch.float64 or not b.is_cuda or not b.is_contiguous()
                                  or b.numel() != int(np.prod(self.data_shape))):
                raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of shape {self.data_shape}")
        self._check_tensor(f, self.data_shape, "f")
        if warm is not None:
            self._check_tensor(warm, self.image_shape, "warm")
        if out is None:
            out = torch.empty(self.image_shape, device=f.device, dtype=torch.float32)
        P = _lib.SolveParams(float(lam), int(outer), int(inner), int(prox_iters), float(L), int(power_iters),
                             int(seed), float(step_scale), int(max_backtrack), int(stall),
                             b_in.data_ptr() if b_in is not None else None,
                             b_out.data_ptr() if b_out is not None else None)
        R = _lib.SolveReport()
        _lib.check(_lib.load().pat_bregman_solve(self._h, f.data_ptr(), warm.data_ptr() if warm is not None else None,
                                                 out.data_ptr(), ctypes.byref(P), ctypes.byref(R),
                                                 _stream_ptr(f.device)))
        rep = {"L": R.L, "inner_total": R.inner_total, "restarts": R.restarts, "energy": R.energy,
               "residuals": [R.residual[i] for i in range(R.n_residual)]}
        return out, rep

    # ------------------------------------------------------------------ device status
    def device_status(self, device=None) -> None:
        """Raise if a bounded device-side wait of this grid's kernels gave up since the last check
        (see pat_device_status); synchronises the current stream of `device`."""
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        _lib.check(_lib.load().pat_device_status(self._h, _stream_ptr(dev)))

    # ------------------------------------------------------------------ kernel timing
    def profile(self, enable: bool = True) -> None:
        """Bracket every kernel launch with CUDA events (see pat_profile_enable)."""
        _lib.check(_lib.load().pat_profile_enable(self._h, int(enable)))

    def profile_read(self) -> dict:
        """{kernel class: (total ms, launches)} since profile(True); waits for the events."""
        n = 16
        names = ctypes.create_string_buffer(48 * n)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        k = ctypes.c_int32()
        _lib.check(_lib.load().pat_profile_read(self._h, n, names, ms, cnt, ctypes.byref(k)))
        out = {}
        for i in range(k.value):
            nm = names.raw[48 * i:48 * (i + 1)].split(b"\0", 1)[0].decode()
            out[nm] = (ms[i], cnt[i])
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().pat_destroy_grid(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

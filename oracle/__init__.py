"""FP64 CPU oracle for the PAT operators A, A^T and C (arXiv:1605.00133).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's CPU-baseline leg are
the only users.  The library in `paper_1605_00133_gb300` never imports this package, and this
package never imports the library; both may be fed from `paper_1605_00133_gb300.synth`, which
holds inputs only.

The arithmetic lives in `pat_oracle.c` (plain C, double precision, its own radix-2 FFT); this
module only marshals numpy arrays through ctypes.  Functions follow the paper as follows:
  forward_plane  A, Sec. 4.3 (k-space pseudospectral time stepping to the detection plane)
  adjoint_plane  A^T, Sec. 4.3-4.4 (transpose; the data act as a time-dependent source)
  sample         C per time point, Sec. 3.1 / Sec. 4.3 (rSP row selection, sHd via FWHT)
  sample_T       C^T
  forward        C A  (Eq. "Fwd" without noise)
  adjoint        A^T C^T (Eq. "BP", back-projection)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pat_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KIND_FULL, KIND_RSP, KIND_SHD01, KIND_SHDPM = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile pat_oracle.c into liboracle.so (gcc, OpenMP, no architecture-specific flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrGrid(ctypes.Structure):
    _fields_ = [("nz", ctypes.c_int32), ("ny", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("dx", ctypes.c_double), ("c", ctypes.c_double), ("rho0", ctypes.c_double),
                ("dt", ctypes.c_double), ("T", ctypes.c_int32), ("pml_size", ctypes.c_int32),
                ("pml_alpha", ctypes.c_double), ("sensor_z", ctypes.c_int32)]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            gp = ctypes.POINTER(OrGrid)
            L.or_forward.argtypes = [gp, _dp, _dp]
            L.or_adjoint.argtypes = [gp, _dp, _dp]
            L.or_fft1.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
            L.or_fft3.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.or_derivative.argtypes = [gp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.or_wavenumber.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
            L.or_wavenumber.restype = ctypes.c_double
            L.or_kappa.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.or_kappa.restype = ctypes.c_double
            L.or_pml_factor.argtypes = [gp, ctypes.c_double, ctypes.c_int]
            L.or_pml_factor.restype = ctypes.c_double
            L.or_fwht.argtypes = [_dp, ctypes.c_int]
            L.or_sample_rsp.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _ip, _dp]
            L.or_sample_rsp_T.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _ip, _dp]
            L.or_sample_shd.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _ip, _ip,
                                        ctypes.c_int, _dp]
            L.or_sample_shd_T.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _ip, _ip,
                                          ctypes.c_int, _dp]
            L.or_num_threads.restype = ctypes.c_int
            L.or_set_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


def or_grid(g) -> OrGrid:
    """OrGrid from any object with the Grid attributes (nz, ny, nx, dx, c, rho0, dt, T, ...)."""
    return OrGrid(g.nz, g.ny, g.nx, g.dx, g.c, g.rho0, g.dt, g.T, g.pml_size, g.pml_alpha,
                  g.sensor_z)


def num_threads() -> int:
    return lib().or_num_threads()


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


# ---------------------------------------------------------------- building blocks (for pins)

def fft1(x, inverse=False):
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    lib().or_fft1(a.ctypes.data, a.size, int(inverse))
    return a


def fft3(x, inverse=False):
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    nz, ny, nx = a.shape
    lib().or_fft3(a.ctypes.data, nz, ny, nx, int(inverse))
    return a


def derivative(g, f, axis, s, transpose=False):
    f = _d(f)
    out = np.empty_like(f)
    gs = or_grid(g)
    lib().or_derivative(ctypes.byref(gs), _ptr(f), _ptr(out), axis, s, int(transpose))
    return out


def wavenumber(m, n, dx):
    return lib().or_wavenumber(m, n, dx)


def kappa(kabs, c, dt):
    return lib().or_kappa(kabs, c, dt)


def pml_factor(g, pos, n):
    gs = or_grid(g)
    return lib().or_pml_factor(ctypes.byref(gs), float(pos), int(n))


def fwht(v):
    a = _d(v).copy()
    lib().or_fwht(_ptr(a), a.size)
    return a


# ---------------------------------------------------------------- operators

def forward_plane(g, p0):
    """A: p0 [Nz][Ny][Nx] -> detection-plane series [T][Ny*Nx]."""
    p0 = _d(p0).reshape(g.nz, g.ny, g.nx)
    out = np.empty((g.T, g.ny * g.nx))
    gs = or_grid(g)
    if lib().or_forward(ctypes.byref(gs), _ptr(p0), _ptr(out)) != 0:
        raise ValueError("oracle: invalid grid")
    return out


def adjoint_plane(g, pbar):
    """A^T: plane series [T][Ny*Nx] -> image [Nz][Ny][Nx]."""
    pbar = _d(pbar).reshape(g.T, g.ny * g.nx)
    out = np.empty((g.nz, g.ny, g.nx))
    gs = or_grid(g)
    if lib().or_adjoint(ctypes.byref(gs), _ptr(pbar), _ptr(out)) != 0:
        raise ValueError("oracle: invalid grid")
    return out


def sample(s, pbar):
    """C per time point: [T][M] -> [T][M_c]."""
    pbar = _d(pbar)
    T, M = pbar.shape
    if s.kind == KIND_FULL:
        return pbar.copy()
    out = np.empty((T, s.m))
    if s.kind == KIND_RSP:
        idx = _i(s.indices)
        lib().or_sample_rsp(T, M, _ptr(pbar), s.m, _ptr(idx, _ip), _ptr(out))
    else:
        perm, rows = _i(s.perm), _i(s.rows)
        lib().or_sample_shd(T, M, _ptr(pbar), s.m, _ptr(perm, _ip), _ptr(rows, _ip),
                            int(s.kind == KIND_SHDPM), _ptr(out))
    return out


def sample_T(s, f, M):
    """C^T per time point: [T][M_c] -> [T][M]."""
    f = _d(f)
    T = f.shape[0]
    if s.kind == KIND_FULL:
        return f.copy()
    out = np.empty((T, M))
    if s.kind == KIND_RSP:
        idx = _i(s.indices)
        lib().or_sample_rsp_T(T, M, _ptr(f), s.m, _ptr(idx, _ip), _ptr(out))
    else:
        perm, rows = _i(s.perm), _i(s.rows)
        lib().or_sample_shd_T(T, M, _ptr(f), s.m, _ptr(perm, _ip), _ptr(rows, _ip),
                              int(s.kind == KIND_SHDPM), _ptr(out))
    return out


def forward(g, s, p0):
    """C A p0 (noise-free data, Eq. "Fwd")."""
    return sample(s, forward_plane(g, p0))


def adjoint(g, s, f):
    """A^T C^T f (back-projection, Eq. "BP")."""
    return adjoint_plane(g, sample_T(s, f, g.ny * g.nx))

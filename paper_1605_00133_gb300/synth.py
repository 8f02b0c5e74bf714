"""Seeded synthetic inputs for compressed-sensing PAT (Arridge et al., arXiv:1605.00133).

This module produces inputs only: pseudo-random numbers, phantoms (initial pressures p0),
sub-sampling index sets and additive noise.  It holds none of the method's arithmetic (no wave
propagation, no FFT, no sampling operator), so both the CUDA path and the FP64 oracle can be fed
from it without sharing any computation.

Random-number generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014).  It is counter based: output k of a stream with seed s is
mix(s + (k+1)*0x9E3779B97F4A7C15), with
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31.
Uniform doubles are (x >> 11) * 2^-53 in [0, 1); integers in [0, n) are floor(u * n); Gaussians
use Box-Muller, sqrt(-2 ln(1-u1)) * cos(2 pi u2).

Seed offsets used by the presets: mask `seed`, scramble permutation `seed+1`, Hadamard rows
`seed+2`, phantom `seed+3`, noise `seed+4`.

Paper passages the inputs imitate:
  * rSP sub-sampling picks M_c random points of the M detection-plane points (Sec. 3.1.1).
  * sHd sub-sampling uses M_c rows of a scrambled Hadamard matrix (Sec. 3.1.2, Sec. 4.3).
  * p0 values lie in [0, 1]: vessels 1, other tissue less (Sec. 5.1); the paper's vascular phantom
    is replaced by seeded branching tubes of the same value range.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of the SplitMix64 stream started at `seed` (uint64)."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK64) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class Stream:
    """Sequential reader over one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed) & _MASK64
        self.pos = 0

    def raw(self, n: int) -> np.ndarray:
        out = splitmix64(self.seed, n, self.pos)
        self.pos += n
        return out

    def uniform(self, n: int = 1) -> np.ndarray:
        """n doubles in [0, 1)."""
        return (self.raw(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def integers(self, n_max: int, n: int = 1) -> np.ndarray:
        """n integers in [0, n_max)."""
        return np.floor(self.uniform(n) * n_max).astype(np.int64)

    def normal(self, n: int = 1) -> np.ndarray:
        """n standard normals by Box-Muller (one pair of uniforms per value)."""
        u = self.uniform(2 * n).reshape(n, 2)
        return np.sqrt(-2.0 * np.log(1.0 - u[:, 0])) * np.cos(2.0 * math.pi * u[:, 1])


def fisher_yates(m: int, seed: int) -> np.ndarray:
    """Seeded Fisher-Yates shuffle of 0..m-1: for i = m-1 down to 1 swap a[i], a[j], j in [0, i]."""
    a = np.arange(m, dtype=np.int64)
    s = Stream(seed)
    u = s.uniform(max(m - 1, 0))
    for t, i in enumerate(range(m - 1, 0, -1)):
        j = int(u[t] * (i + 1))
        a[i], a[j] = a[j], a[i]
    return a


# --------------------------------------------------------------------------------------------
# Sub-sampling index sets (Sec. 3.1)
# --------------------------------------------------------------------------------------------

def rsp_indices(m_plane: int, m_c: int, seed: int) -> np.ndarray:
    """rSP: M_c distinct plane points = first M_c of a seeded shuffle, sorted ascending (int32).

    Linear plane index is y * Nx + x.
    """
    if not 0 <= m_c <= m_plane:
        raise ValueError("need 0 <= m_c <= m_plane")
    return np.sort(fisher_yates(m_plane, seed)[:m_c]).astype(np.int32)


def shd_pattern(m_plane: int, m_c: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """sHd: (scramble permutation pi of the M plane points, selected Hadamard rows R).

    pi = shuffle(seed + 1); R = first M_c of shuffle(seed + 2), kept in draw order.
    M must be a power of two (Sylvester Hadamard order).
    """
    if m_plane & (m_plane - 1):
        raise ValueError("sHd needs a power-of-two plane size")
    if not 0 <= m_c <= m_plane:
        raise ValueError("need 0 <= m_c <= m_plane")
    perm = fisher_yates(m_plane, seed + 1).astype(np.int32)
    rows = fisher_yates(m_plane, seed + 2)[:m_c].astype(np.int32)
    return perm, rows


def gsp_indices(ny: int, nx: int, step: int, offset: int = 0) -> np.ndarray:
    """Regular coarse grid of plane points (gSP / regular sub-grid, Sec. 5.3), ascending int32."""
    ys = np.arange(offset, ny, step)
    xs = np.arange(offset, nx, step)
    return (ys[:, None] * nx + xs[None, :]).ravel().astype(np.int32)


# --------------------------------------------------------------------------------------------
# Phantoms (initial pressure p0), layout [Nz][Ny][Nx], z = depth
# --------------------------------------------------------------------------------------------

def _interior_box(shape, pml, margin):
    lo = np.array([pml + margin] * 3, dtype=np.float64)
    hi = np.array([n - 1 - pml - margin for n in shape], dtype=np.float64)
    return lo, hi


def gaussian_balls(shape, n_balls: int, sigma: float, seed: int, pml: int = 0,
                   amp_range=(0.5, 1.0)) -> np.ndarray:
    """Sum of isotropic Gaussian balls exp(-|r-c|^2/(2 sigma^2)), amplitudes U[amp_range].

    Centres are uniform in the interior, at least 2 sigma away from the absorbing layer.
    """
    s = Stream(seed)
    lo, hi = _interior_box(shape, pml, 2.0 * sigma)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    p0 = np.zeros(shape, dtype=np.float64)
    for _ in range(n_balls):
        c = lo + s.uniform(3) * (hi - lo)
        a = amp_range[0] + s.uniform(1)[0] * (amp_range[1] - amp_range[0])
        r2 = (z - c[0]) ** 2 + (y - c[1]) ** 2 + (x - c[2]) ** 2
        p0 += a * np.exp(-r2 / (2.0 * sigma * sigma))
    return p0


def radial_gaussian(shape, centre, sigma: float, amp: float = 1.0) -> np.ndarray:
    """A single radially symmetric Gaussian amp*exp(-r^2/(2 sigma^2)) about `centre` (z,y,x)."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (z - centre[0]) ** 2 + (y - centre[1]) ** 2 + (x - centre[2]) ** 2
    return amp * np.exp(-r2 / (2.0 * sigma * sigma))


def _gauss_smooth(vol: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian smoothing (truncated at 3 sigma, zero outside the volume)."""
    if sigma <= 0:
        return vol
    r = int(math.ceil(3 * sigma))
    t = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-t * t / (2 * sigma * sigma))
    k /= k.sum()
    out = vol
    for ax in range(3):
        padw = [(0, 0)] * 3
        padw[ax] = (r, r)
        pv = np.pad(out, padw)
        acc = np.zeros_like(out)
        n = out.shape[ax]
        for i, w in enumerate(k):
            sl = [slice(None)] * 3
            sl[ax] = slice(i, i + n)
            acc += w * pv[tuple(sl)]
        out = acc
    return out


def _paint_capsule(vol, a, b, radius, value):
    """vol = max(vol, value) on voxels within `radius` of segment a-b (coords z,y,x)."""
    lo = np.floor(np.minimum(a, b) - radius - 1).astype(int)
    hi = np.ceil(np.maximum(a, b) + radius + 1).astype(int)
    lo = np.maximum(lo, 0)
    hi = np.minimum(hi, np.array(vol.shape) - 1)
    if np.any(hi < lo):
        return
    zz, yy, xx = np.meshgrid(np.arange(lo[0], hi[0] + 1), np.arange(lo[1], hi[1] + 1),
                             np.arange(lo[2], hi[2] + 1), indexing="ij")
    pts = np.stack([zz, yy, xx], axis=-1).astype(np.float64)
    d = b - a
    L2 = float(d @ d)
    if L2 == 0.0:
        t = np.zeros(pts.shape[:-1])
    else:
        t = np.clip(((pts - a) @ d) / L2, 0.0, 1.0)
    proj = a + t[..., None] * d
    dist2 = np.sum((pts - proj) ** 2, axis=-1)
    inside = dist2 <= radius * radius
    sub = vol[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1, lo[2]:hi[2] + 1]
    np.maximum(sub, np.where(inside, value, 0.0), out=sub)


def branching_tubes(shape, n_tubes: int, seed: int, pml: int = 0, radius_range=(1.0, 4.0),
                    seg_len=(8.0, 24.0), branch_prob: float = 0.3, jitter: float = 0.35,
                    max_segments: int = 6, smooth_sigma: float = 1.0) -> np.ndarray:
    """Seeded vessel-like phantom: random-walk centre lines with branches, values in [0, 1].

    Each tube: start uniform in the interior, random unit direction, up to `max_segments`
    segments of length U[seg_len]; each segment end spawns a side branch with probability
    `branch_prob`; directions get Gaussian jitter.  Radius U[radius_range] and value U[0, 1]
    per tube; tubes are max-combined, Gaussian-smoothed (sigma 1 voxel), clamped to [0, 1]
    and zeroed in the absorbing layer.
    """
    s = Stream(seed)
    rmax = radius_range[1]
    lo, hi = _interior_box(shape, pml, rmax + 1.0)
    vol = np.zeros(shape, dtype=np.float64)

    def unit(v):
        n = np.linalg.norm(v)
        return v / n if n > 0 else np.array([0.0, 0.0, 1.0])

    for _ in range(n_tubes):
        radius = radius_range[0] + s.uniform(1)[0] * (radius_range[1] - radius_range[0])
        value = s.uniform(1)[0]
        start = lo + s.uniform(3) * (hi - lo)
        stack = [(start, unit(s.normal(3)), max_segments)]
        while stack:
            pos, direc, left = stack.pop()
            for _seg in range(left):
                length = seg_len[0] + s.uniform(1)[0] * (seg_len[1] - seg_len[0])
                direc = unit(direc + jitter * s.normal(3))
                end = np.clip(pos + length * direc, lo, hi)
                _paint_capsule(vol, pos, end, radius, value)
                if s.uniform(1)[0] < branch_prob and left > 1:
                    stack.append((end.copy(), unit(direc + 1.0 * s.normal(3)), left // 2))
                pos = end
    vol = np.clip(_gauss_smooth(vol, smooth_sigma), 0.0, 1.0)
    if pml > 0:
        vol[:pml] = 0; vol[-pml:] = 0
        vol[:, :pml] = 0; vol[:, -pml:] = 0
        vol[:, :, :pml] = 0; vol[:, :, -pml:] = 0
    return vol


# --------------------------------------------------------------------------------------------
# Noise
# --------------------------------------------------------------------------------------------

def band_limit(vol: np.ndarray) -> np.ndarray:
    """vol with its Nyquist planes removed (the field's spectrum then lies strictly inside the grid's
    band, so it is represented identically on any finer grid)."""
    F = np.fft.fftn(vol)
    for ax, n in enumerate(vol.shape):
        idx = [slice(None)] * vol.ndim
        idx[ax] = n // 2
        F[tuple(idx)] = 0.0
    return np.fft.ifftn(F).real


def upsample2(vol: np.ndarray) -> np.ndarray:
    """The band-limited (trigonometric) interpolant of vol on the grid with half the spacing: equal to
    vol at the coincident points [::2, ::2, ::2].  vol must have no Nyquist content (band_limit)."""
    F = np.fft.fftn(vol)
    shape2 = tuple(2 * n for n in vol.shape)
    G = np.zeros(shape2, dtype=complex)
    sl = [np.r_[0:n // 2, n * 2 - n // 2:n * 2] for n in vol.shape]
    src = [np.r_[0:n // 2, n - n // 2:n] for n in vol.shape]
    G[np.ix_(*sl)] = F[np.ix_(*src)]
    return np.fft.ifftn(G).real * 8.0


def gaussian_noise(shape, sigma: float, seed: int) -> np.ndarray:
    """i.i.d. N(0, sigma^2) noise of the given shape."""
    n = int(np.prod(shape))
    return sigma * Stream(seed).normal(n).reshape(shape)


def add_relative_noise(f: np.ndarray, rel: float, seed: int) -> np.ndarray:
    """f + noise with sigma = rel * max|f| (the configs' "1% Gaussian noise")."""
    sigma = rel * float(np.max(np.abs(f))) if f.size else 0.0
    return f + gaussian_noise(f.shape, sigma, seed)

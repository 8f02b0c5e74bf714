"""Grid / sampling presets for the five workloads this library is measured on.

Physical model (Sec. 4.3 and Table 2 of arXiv:1605.00133): homogeneous sound speed c, isotropic
voxel size dx, time step dt = cfl * dx / c, recording at every time step (Delta_t = delta_t).
Grid layout is (Nz, Ny, Nx) with z the depth axis (the paper's x) and the detection plane at
z = sensor_z.  The absorbing layer (PML) lies inside the grid on all six faces; the detection
plane is its first interior layer.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

from . import synth

# sampling kinds (same values as pat_sampling_kind in include/pat.h)
KIND_FULL = 0      # conventional: every plane point, data [T][Ny*Nx]
KIND_RSP = 1       # random single points (or any index list, e.g. a regular gSP grid)
KIND_SHD01 = 2     # scrambled Hadamard, 0/1 patterns (as a DMD realises them)
KIND_SHDPM = 3     # scrambled Hadamard, +-1/sqrt(M) patterns (orthonormal rows)


@dataclass
class Grid:
    nz: int
    ny: int
    nx: int
    dx: float = 100e-6
    c: float = 1500.0
    rho0: float = 1.0
    cfl: float = 0.3
    dt: float = 0.0            # <= 0: cfl * dx / c
    T: int = 64                # recorded samples n = 0..T-1
    pml_size: int = 8
    pml_alpha: float = 2.0
    sensor_z: int = -1         # < 0: pml_size
    batch: int = 1

    def __post_init__(self):
        if self.dt <= 0:
            self.dt = self.cfl * self.dx / self.c
        if self.sensor_z < 0:
            self.sensor_z = self.pml_size

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def n(self):
        return self.nz * self.ny * self.nx

    @property
    def m_plane(self):
        return self.ny * self.nx


@dataclass
class Sampling:
    kind: int = KIND_FULL
    m: int = 0                       # M_c (KIND_FULL: Ny*Nx)
    indices: "object" = None         # int32[M_c] plane indices (KIND_RSP)
    perm: "object" = None            # int32[M] scramble permutation (sHd)
    rows: "object" = None            # int32[M_c] Hadamard rows (sHd)


@dataclass
class Workload:
    name: str
    grid: Grid
    sampling: Sampling
    phantom: str
    seed: int = 0
    noise_rel: float = 0.01
    bregman_outer: int = 5
    inner: int = 20
    extra: dict = field(default_factory=dict)

    def p0(self, seed_offset: int = 0):
        g = self.grid
        s = self.seed + 3 + seed_offset
        if self.phantom == "balls3":
            return synth.gaussian_balls(g.shape, 3, 2.0, s, pml=g.pml_size)
        if self.phantom.startswith("tubes"):
            return synth.branching_tubes(g.shape, int(self.phantom[5:]), s, pml=g.pml_size)
        raise ValueError(self.phantom)


def make_sampling(grid: Grid, kind: int, m_c: int, seed: int) -> Sampling:
    M = grid.m_plane
    if kind == KIND_FULL:
        return Sampling(KIND_FULL, M)
    if kind == KIND_RSP:
        return Sampling(KIND_RSP, m_c, indices=synth.rsp_indices(M, m_c, seed))
    if kind in (KIND_SHD01, KIND_SHDPM):
        perm, rows = synth.shd_pattern(M, m_c, seed)
        return Sampling(kind, m_c, perm=perm, rows=rows)
    raise ValueError(kind)


def workload(name: str, seed: int = 0) -> Workload:
    """Named workloads.

    c1  32^3, dx 100 um, c 1500, CFL 0.3, T 64, 8-pt PML, 3 Gaussian balls, rSP 25 %.
    c2  64x128x128, dx 100 um, T 400, 10-pt PML, 20 branching tubes, rSP 12.5 % (2048/16384).
    c3  c2 grid with scrambled-Hadamard 0/1 patterns, m = 2048 of 16384.
    c4  128x256x256, dx 50 um, T 800, 10-pt PML, 60 tubes, rSP 1/16 (4096/65536).
    c2gsp  c2 with regular-grid single points, gSP-16 (every 4th point in y and x: 1024/16384).
    """
    if name == "c1":
        g = Grid(32, 32, 32, dx=100e-6, T=64, pml_size=8)
        return Workload(name, g, make_sampling(g, KIND_RSP, 256, seed), "balls3", seed,
                        bregman_outer=5, inner=20)
    if name == "c2":
        g = Grid(64, 128, 128, dx=100e-6, T=400, pml_size=10)
        return Workload(name, g, make_sampling(g, KIND_RSP, 2048, seed), "tubes20", seed,
                        bregman_outer=5, inner=50)
    if name == "c3":
        g = Grid(64, 128, 128, dx=100e-6, T=400, pml_size=10)
        return Workload(name, g, make_sampling(g, KIND_SHD01, 2048, seed), "tubes20", seed,
                        bregman_outer=5, inner=50)
    if name == "c4":
        g = Grid(128, 256, 256, dx=50e-6, T=800, pml_size=10)
        return Workload(name, g, make_sampling(g, KIND_RSP, 4096, seed), "tubes60", seed,
                        bregman_outer=5, inner=50)
    if name == "c2gsp":
        g = Grid(64, 128, 128, dx=100e-6, T=400, pml_size=10)
        s = Sampling(KIND_RSP, 1024, indices=synth.gsp_indices(g.ny, g.nx, 4))
        return Workload(name, g, s, "tubes20", seed, bregman_outer=5, inner=50)
    raise ValueError(f"unknown workload {name!r}")


def shrink(w: Workload, T: int) -> Workload:
    """Same workload with fewer recorded samples (for bounded CPU samples and quick tests)."""
    return replace(w, grid=replace(w.grid, T=T))

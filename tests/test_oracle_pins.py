"""Pins of the FP64 oracle against facts fixed outside it (no GPU).

Each test checks the oracle against mathematics or the paper, never against itself:
brute-force DFT and dense Hadamard matrices, the exact per-mode solution of the k-space scheme,
the d'Alembert spherical wave, a dense-matrix transpose on a tiny grid, and dot-product tests.
"""
import math

import numpy as np
import pytest

from paper_1605_00133_gb300 import presets, synth


# ------------------------------------------------------------------------------- FFT

def dft_matrix(n, inverse=False):
    j = np.arange(n)
    s = 1.0 if inverse else -1.0
    W = np.exp(s * 2j * np.pi * np.outer(j, j) / n)
    return W / n if inverse else W


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64])
def test_fft1_matches_brute_force_dft(oracle_mod, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    np.testing.assert_allclose(oracle_mod.fft1(x), dft_matrix(n) @ x, rtol=0, atol=1e-13 * n)
    np.testing.assert_allclose(oracle_mod.fft1(x, inverse=True), dft_matrix(n, True) @ x,
                               rtol=0, atol=1e-14 * n)


def test_fft1_round_trip_and_parseval(oracle_mod):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(256) + 1j * rng.standard_normal(256)
    X = oracle_mod.fft1(x)
    assert np.abs(oracle_mod.fft1(X, inverse=True) - x).max() < 1e-14
    assert abs(np.vdot(X, X).real / 256 - np.vdot(x, x).real) < 1e-12 * np.vdot(x, x).real


def test_fft3_is_separable_dft(oracle_mod):
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 8, 16)) + 1j * rng.standard_normal((4, 8, 16))
    ref = np.einsum("az,by,cx,zyx->abc", dft_matrix(4), dft_matrix(8), dft_matrix(16), x)
    np.testing.assert_allclose(oracle_mod.fft3(x), ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle_mod.fft3(oracle_mod.fft3(x), inverse=True), x, atol=1e-14)


# ------------------------------------------------------------------------------- k-space pieces

def test_wavenumber_and_kappa(oracle_mod):
    dx = 1e-4
    # bins 0..n/2-1 positive, Nyquist and above negative
    assert oracle_mod.wavenumber(0, 8, dx) == 0.0
    assert oracle_mod.wavenumber(1, 8, dx) == pytest.approx(2 * math.pi / (8 * dx))
    assert oracle_mod.wavenumber(4, 8, dx) == pytest.approx(-math.pi / dx)
    assert oracle_mod.wavenumber(7, 8, dx) == pytest.approx(-2 * math.pi / (8 * dx))
    assert oracle_mod.kappa(0.0, 1500.0, 2e-8) == 1.0
    k = 1234.5
    x = 0.5 * 1500.0 * 2e-8 * k
    assert oracle_mod.kappa(k, 1500.0, 2e-8) == pytest.approx(math.sin(x) / x, rel=1e-15)


def test_derivative_of_a_plane_wave(oracle_mod):
    """D^+ of cos(k x) on a periodic grid is -k kappa sin(k (x + dx/2)) (phase shift +dx/2)."""
    g = presets.Grid(8, 8, 16, pml_size=0, sensor_z=0)
    kx = 2 * math.pi * 3 / (16 * g.dx)
    x = np.arange(16) * g.dx
    f = np.broadcast_to(np.cos(kx * x), g.shape).copy()
    kap = math.sin(0.5 * g.c * g.dt * kx) / (0.5 * g.c * g.dt * kx)
    got_p = oracle_mod.derivative(g, f, 2, +1)
    got_m = oracle_mod.derivative(g, f, 2, -1)
    np.testing.assert_allclose(got_p[0, 0], -kx * kap * np.sin(kx * (x + g.dx / 2)), atol=1e-9 * kx)
    np.testing.assert_allclose(got_m[0, 0], -kx * kap * np.sin(kx * (x - g.dx / 2)), atol=1e-9 * kx)
    # other axes see a constant
    assert np.abs(oracle_mod.derivative(g, f, 0, +1)).max() < 1e-9 * kx


def test_pml_profile(oracle_mod):
    g = presets.Grid(32, 32, 32, pml_size=8, pml_alpha=2.0)
    n, P = 32, 8
    # interior untouched
    for pos in [8.0, 15.5, 23.0]:
        assert oracle_mod.pml_factor(g, pos, n) == 1.0
    # full depth: alpha = pml_alpha * c/dx, factor exp(-alpha dt/2) = exp(-pml_alpha * cfl / 2)
    assert oracle_mod.pml_factor(g, 0.0, n) == pytest.approx(math.exp(-2.0 * 0.3 / 2), rel=1e-14)
    assert oracle_mod.pml_factor(g, 31.0, n) == pytest.approx(math.exp(-2.0 * 0.3 / 2), rel=1e-14)
    # fourth-order profile at depth 4 of 8
    assert oracle_mod.pml_factor(g, 4.0, n) == pytest.approx(math.exp(-0.3 * (0.5 ** 4)), rel=1e-14)
    # staggered point j + 1/2 = 7.5 sits 1/2 voxel into the layer
    assert oracle_mod.pml_factor(g, 7.5, n) == pytest.approx(math.exp(-0.3 * (0.5 / P) ** 4), rel=1e-14)


# ------------------------------------------------------------------------------- physics pins

def spectral_solution(g, p0, n):
    """p^n = F^-1[ cos(n c |k| dt) F p0 ]: exact solution of the periodic k-space scheme."""
    ks = []
    for m in g.shape:
        k = 2 * np.pi * np.fft.fftfreq(m, g.dx)
        ks.append(k)
    K = np.sqrt(ks[0][:, None, None] ** 2 + ks[1][None, :, None] ** 2 + ks[2][None, None, :] ** 2)
    return np.real(np.fft.ifftn(np.fft.fftn(p0) * np.cos(n * g.c * K * g.dt)))


@pytest.mark.parametrize("shape", [(8, 8, 8), (16, 8, 32), (16, 16, 16)])
def test_forward_matches_exact_spectral_solution_without_pml(oracle_mod, shape):
    """PML off: eliminating u gives p^{n+1} - 2 p^n + p^{n-1} = -4 sin^2(c|k|dt/2) p^n per mode, and
    the half-step start gives p^1 = cos(c|k|dt) p^0, so p^n = cos(n c|k| dt) p0 exactly."""
    g = presets.Grid(*shape, T=24, pml_size=0, sensor_z=shape[0] // 3)
    p0 = np.random.default_rng(3).standard_normal(shape)
    pbar = oracle_mod.forward_plane(g, p0)
    scale = np.abs(p0).max()
    for n in range(g.T):
        ref = spectral_solution(g, p0, n)[g.sensor_z].ravel()
        assert np.abs(pbar[n] - ref).max() < 1e-12 * scale, n
    # recorded sample 0 is p0 itself on the plane (Eq. PATfwd initial condition)
    assert np.array_equal(pbar[0], p0[g.sensor_z].ravel())


def dalembert_gaussian(r, t, c, sigma, amp):
    """Free-space solution of Eq. PATfwd for p0(r) = amp exp(-r^2/(2 sigma^2)), dp/dt(0) = 0:
    p(r,t) = [(r - ct) p0(r - ct) + (r + ct) p0(r + ct)] / (2 r), p0 extended evenly."""
    p0 = lambda s: amp * np.exp(-s * s / (2 * sigma * sigma))
    a, b = r - c * t, r + c * t
    return (a * p0(a) + b * p0(b)) / (2 * r)


def spherical_case(oracle_mod, pml_size, T):
    g = presets.Grid(32, 32, 32, T=T, pml_size=pml_size, sensor_z=8)
    centre = (16.0, 16.0, 16.0)
    sigma = 2.0
    p0 = synth.radial_gaussian(g.shape, centre, sigma)
    pbar = oracle_mod.forward_plane(g, p0)
    yy, xx = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    # without the PML the grid is periodic: sum the free-space waves of the nearest images
    shifts = [-32, 0, 32] if pml_size == 0 else [0]
    ref = np.zeros((T, 32 * 32))
    for sz in shifts:
        for sy in shifts:
            for sx in shifts:
                r = np.sqrt((g.sensor_z - centre[0] - sz) ** 2 + (yy - centre[1] - sy) ** 2
                            + (xx - centre[2] - sx) ** 2)
                ref += np.stack([dalembert_gaussian(r * g.dx, n * g.dt, g.c, sigma * g.dx, 1.0).ravel()
                                 for n in range(T)])
    return g, pbar, ref


def test_spherical_wave_without_pml(oracle_mod):
    """Radially symmetric Gaussian (sigma = 2 voxels) in a homogeneous medium.  Without the PML the
    grid is periodic, so the reference is the d'Alembert solution summed over the 27 nearest periodic
    images.  The scheme is exact per Fourier mode, so what remains is the Gaussian's content beyond
    the grid's Nyquist frequency, ~exp(-(pi sigma)^2/2) ~ 3e-9."""
    g, pbar, ref = spherical_case(oracle_mod, 0, 60)
    err = np.linalg.norm(pbar - ref) / np.linalg.norm(ref)
    assert err < 1e-9, err


def test_spherical_wave_with_pml(oracle_mod):
    """Same wave with the 8-voxel PML on all faces: the absorbing layer begins right behind the
    detection plane, so the trace differs from free space only by the layer's reflection."""
    g, pbar, ref = spherical_case(oracle_mod, 8, 60)
    inner = np.zeros((32, 32), bool)
    inner[8:24, 8:24] = True
    inner = inner.ravel()
    # plane points outside the lateral layers; measured reflection level ~1e-5 by ct = 18 voxels
    err = np.linalg.norm(pbar[:, inner] - ref[:, inner]) / np.linalg.norm(ref[:, inner])
    assert err < 1e-4, err


def test_forward_commutes_with_lateral_shift_without_pml(oracle_mod):
    """Periodic, homogeneous, PML off: shifting p0 in (y, x) shifts the plane series identically."""
    g = presets.Grid(8, 16, 16, T=10, pml_size=0, sensor_z=2)
    p0 = np.random.default_rng(4).standard_normal(g.shape)
    a = oracle_mod.forward_plane(g, p0).reshape(g.T, 16, 16)
    b = oracle_mod.forward_plane(g, np.roll(p0, (3, 5), axis=(1, 2))).reshape(g.T, 16, 16)
    np.testing.assert_allclose(np.roll(a, (3, 5), axis=(1, 2)), b, atol=1e-12)


# ------------------------------------------------------------------------------- adjoint pins

def test_dense_transpose_on_8cubed(oracle_mod):
    """Build A (512 columns) and A^T (T*M columns) on an 8^3 grid with a 2-voxel PML; the adjoint
    routine must be the exact transpose of the forward recurrence."""
    g = presets.Grid(8, 8, 8, T=16, pml_size=2, sensor_z=2)
    N, TM = g.n, g.T * g.m_plane
    A = np.empty((TM, N))
    for j in range(N):
        e = np.zeros(N); e[j] = 1.0
        A[:, j] = oracle_mod.forward_plane(g, e.reshape(g.shape)).ravel()
    At = np.empty((N, TM))
    for j in range(TM):
        e = np.zeros(TM); e[j] = 1.0
        At[:, j] = oracle_mod.adjoint_plane(g, e.reshape(g.T, g.m_plane)).ravel()
    assert np.abs(At - A.T).max() <= 1e-13 * np.abs(A).max()
    # spectral norm of C A by dense SVD is positive and finite (feeds the solver's step size)
    s = np.linalg.svd(A, compute_uv=False)
    assert 0 < s[0] < 10


@pytest.mark.parametrize("name,T,kind", [("c1", 64, presets.KIND_RSP), ("c2", 5, presets.KIND_RSP),
                                         ("c3", 5, presets.KIND_SHD01),
                                         ("c3", 4, presets.KIND_SHDPM)])
def test_dot_product_adjoint(oracle_mod, name, T, kind):
    """|<C A x, y> - <x, A^T C^T y>| / (||C A x|| ||y||) < 1e-12 on the workload shapes."""
    w = presets.shrink(presets.workload(name), T)
    g = w.grid
    s = presets.make_sampling(g, kind, w.sampling.m, 7)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(g.shape)
    y = rng.standard_normal((g.T, s.m))
    Ax = oracle_mod.forward(g, s, x)
    Aty = oracle_mod.adjoint(g, s, y)
    rel = abs(np.sum(Ax * y) - np.sum(x * Aty)) / (np.linalg.norm(Ax) * np.linalg.norm(y))
    assert rel < 1e-12, rel


# ------------------------------------------------------------------------------- sampling pins

def hadamard(m):
    i = np.arange(m)
    pc = np.vectorize(lambda v: bin(v).count("1"))(np.bitwise_and.outer(i, i))
    return np.where(pc % 2 == 0, 1.0, -1.0)


@pytest.mark.parametrize("m", [1, 2, 8, 64, 1024])
def test_fwht_matches_dense_hadamard(oracle_mod, m):
    H = hadamard(m)
    v = np.random.default_rng(m).standard_normal(m)
    np.testing.assert_allclose(oracle_mod.fwht(v), H @ v, atol=1e-12 * m)
    if m <= 64:
        assert np.array_equal(H @ H, m * np.eye(m))
        for i in range(m):  # transform of e_i is row i
            e = np.zeros(m); e[i] = 1.0
            assert np.array_equal(oracle_mod.fwht(e), H[i])


@pytest.mark.parametrize("kind", [presets.KIND_SHD01, presets.KIND_SHDPM])
def test_shd_matches_dense_patterns(oracle_mod, kind):
    """f_j(t) = sum_l phi_j(l) pbar(l, t) with binary (0/1) or +-1/sqrt(M) scrambled Hadamard
    patterns phi_j(perm[l]) = (1 + H[R_j, l])/2 or H[R_j, l]/sqrt(M) (Eq. GenScan, Sec. 4.3)."""
    M, mc, T = 256, 40, 3
    perm, rows = synth.shd_pattern(M, mc, 11)
    H = hadamard(M)
    Phi = np.zeros((mc, M))
    for j in range(mc):
        row = (1 + H[rows[j]]) / 2 if kind == presets.KIND_SHD01 else H[rows[j]] / math.sqrt(M)
        Phi[j, perm] = row
    s = presets.Sampling(kind, mc, perm=perm, rows=rows)
    pbar = np.random.default_rng(6).standard_normal((T, M))
    np.testing.assert_allclose(oracle_mod.sample(s, pbar), pbar @ Phi.T, atol=1e-12)
    f = np.random.default_rng(7).standard_normal((T, mc))
    np.testing.assert_allclose(oracle_mod.sample_T(s, f, M), f @ Phi, atol=1e-12)
    if kind == presets.KIND_SHDPM:  # orthonormal rows: C C^T = I, so C^dagger = C^T (Sec. 4.4)
        np.testing.assert_allclose(Phi @ Phi.T, np.eye(mc), atol=1e-12)


def test_rsp_is_row_selection(oracle_mod):
    M, mc, T = 1024, 256, 4
    idx = synth.rsp_indices(M, mc, 3)
    assert len(np.unique(idx)) == mc and np.all(np.diff(idx) > 0)
    s = presets.Sampling(presets.KIND_RSP, mc, indices=idx)
    pbar = np.random.default_rng(8).standard_normal((T, M))
    f = oracle_mod.sample(s, pbar)
    assert np.array_equal(f, pbar[:, idx])
    back = oracle_mod.sample_T(s, f, M)
    assert np.array_equal(back[:, idx], f) and np.count_nonzero(back) <= T * mc
    # C C^T = I (pseudo-inverse equals transpose, Sec. 4.4)
    assert np.array_equal(oracle_mod.sample(s, oracle_mod.sample_T(s, f, M)), f)


def test_integer_inputs_are_exact_in_shd(oracle_mod):
    """Integer-valued planes give integer (or half-integer) data exactly: the GPU must match bit
    for bit."""
    M, mc = 1024, 100
    perm, rows = synth.shd_pattern(M, mc, 2)
    s = presets.Sampling(presets.KIND_SHD01, mc, perm=perm, rows=rows)
    pbar = np.random.default_rng(9).integers(-50, 50, size=(2, M)).astype(float)
    f = oracle_mod.sample(s, pbar)
    assert np.array_equal(f * 2, np.round(f * 2))

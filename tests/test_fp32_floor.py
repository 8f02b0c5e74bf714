"""Pins of the FP32-floor restatement (tests/fp32_floor.py): in float64 it is the oracle's recurrence
(forward and adjoint agree with the FP64 oracle to rounding), and in float32 it lands where an FP32
evaluation should (far below 1e-5 after a few steps, far above FP64 rounding).  Only then do its
float32 errors at full size say what an FP32 implementation of the scheme can reach."""
import numpy as np
import pytest

from paper_1605_00133_gb300 import presets

import fp32_floor as ff  # noqa: E402

SHAPES = [(16, 32, 16), (8, 16, 32)]


@pytest.mark.parametrize("shape", SHAPES)
def test_float64_restatement_is_the_oracle(oracle_mod, shape):
    g = presets.Grid(*shape, T=20, pml_size=3, sensor_z=4)
    sc = ff.Scheme(g, np.float64, workers=1)
    rng = np.random.default_rng(31)
    p0 = rng.standard_normal(g.shape)
    assert ff.rel(sc.forward_plane(p0), oracle_mod.forward_plane(g, p0)) < 1e-12
    y = rng.standard_normal((g.T, g.m_plane))
    assert ff.rel(sc.adjoint_plane(y), oracle_mod.adjoint_plane(g, y)) < 1e-12


def test_float64_restatement_adjoint_is_the_transpose():
    """<A x, y> = <x, A^T y> in float64, independently of the oracle."""
    g = presets.Grid(8, 16, 16, T=12, pml_size=2)
    sc = ff.Scheme(g, np.float64, workers=1)
    rng = np.random.default_rng(32)
    x = rng.standard_normal(g.shape)
    y = rng.standard_normal((g.T, g.m_plane))
    lhs = np.sum(sc.forward_plane(x) * y)
    rhs = np.sum(x * sc.adjoint_plane(y))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs) + 1e-12


def test_float32_restatement_error_is_fp32_rounding(oracle_mod):
    g = presets.Grid(16, 32, 16, T=20, pml_size=3)
    rng = np.random.default_rng(33)
    p0 = rng.standard_normal(g.shape)
    y = rng.standard_normal((g.T, g.m_plane))
    sc = ff.Scheme(g, np.float32, workers=1)
    ef = ff.rel(sc.forward_plane(p0), oracle_mod.forward_plane(g, p0))
    ea = ff.rel(sc.adjoint_plane(y), oracle_mod.adjoint_plane(g, y))
    for e in (ef, ea):
        assert 1e-9 < e < 2e-6

"""Numbers printed in the paper that the presets' unit conventions must reproduce."""
import json
import math
import os

import pytest

from paper_1605_00133_gb300 import presets

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table2_model_parameters.json")))


def test_tumor1_time_step_is_cfl_0p3():
    """Table 2: dx = 156.25 um, dt = 31.25 ns, c = 1500 m/s -> c dt / dx = 0.3, the CFL number the
    presets use; Grid derives dt = cfl dx / c."""
    t = G["Tumor1"]
    g = presets.Grid(*t["N"], dx=t["dx_um"] * 1e-6, c=t["c0"], cfl=0.3)
    assert g.dt == pytest.approx(t["dt_ns"] * 1e-9, rel=1e-12)


def test_tumor1_mt_crosses_the_cube_diagonal():
    """Mt = 740 = ceil(sqrt(3) * 128 / 0.3): time for a wave to cross the cube's diagonal."""
    t = G["Tumor1"]
    assert math.ceil(math.sqrt(3) * t["N"][0] / 0.3) == t["Mt"]


def test_nyquist_relation():
    """Sec. 2.2: spatial spacing dx resolves temporal frequencies up to c / (2 dx); the Tumor1 grid
    gives the 4.8 MHz band limit quoted in Sec. 5.2."""
    t = G["Tumor1"]
    f = t["c0"] / (2 * t["dx_um"] * 1e-6)
    assert f / 1e6 == pytest.approx(t["band_limit_MHz"], abs=0.05)


def test_hair_twelve_steps():
    """Sec. 6.2: 12 time steps move a wave 12 c dt / dx = 5.8 voxels on the Hair grid."""
    t = G["Hair"]
    v = 12 * t["c0"] * t["dt_ns"] * 1e-9 / (t["dx_um"][0] * 1e-6)
    assert v == pytest.approx(t["twelve_steps_in_voxels"], abs=0.01)


def test_plane_sizes():
    for k in ("Tumor1", "Knot", "Vessels"):
        t = G[k]
        assert t["N"][1] * t["N"][2] >= t["M"] or k == "Vessels"
    assert G["Tumor1"]["M"] == 128 * 128 == presets.workload("c2").grid.m_plane

"""Plug / rupture / aerosol analysis (lbm_plug_analysis) on synthetic fields:
interface positions against the tanh profiles' known midpoints, droplet count
and mass against scipy's connected-component labelling."""
import numpy as np
import pytest

import synth

ndimage = pytest.importorskip("scipy.ndimage")

RL, RG = 0.2793, 0.0316
MID = 0.5 * (RL + RG)


@pytest.fixture(scope="module")
def lbm():
    from paper_2103_08301_gb300 import build
    build.build()
    import paper_2103_08301_gb300 as m
    return m


def _reference(rho, mid):
    ny, nx = rho.shape
    liq = np.zeros_like(rho, dtype=bool)
    liq[1:ny - 1] = rho[1:ny - 1] > mid
    lab, n = ndimage.label(liq)  # 4-connectivity
    drops, dmass, wmass = 0, 0.0, 0.0
    for k in range(1, n + 1):
        m = lab == k
        wall = m[1].any() or m[ny - 2].any()
        if wall:
            wmass += rho[m].sum()
        else:
            drops += 1
            dmass += rho[m].sum()
    intact = bool(liq[1:ny - 1].all(axis=0).any())
    return drops, dmass, wmass, intact


def test_intact_plug_interfaces(lbm):
    nx, ny = 400, 64
    rho = synth.airway_rho0(nx, ny, 5, 120.0, 80.0, RL, RG)
    st = lbm.lbm_plug_analysis(rho, MID)
    assert st["intact"] == 1
    assert abs(st["x_rear"] - 120.0) < 0.05 and abs(st["x_front"] - 200.0) < 0.05
    drops, dmass, wmass, intact = _reference(rho, MID)
    assert st["n_droplets"] == drops == 0
    assert abs(st["wall_liquid_mass"] - wmass) < 1e-9 * wmass


def test_ruptured_plug_with_droplets(lbm):
    nx, ny = 400, 80
    film = synth.airway_rho0(nx, ny, 6, 1e9, 0.0, RL, RG)  # films only
    d1 = synth.disk_rho0(nx, ny, 10, RL, RG, centre=(150.0, 40.0))
    d2 = synth.disk_rho0(nx, ny, 7, RL, RG, centre=(260.0, 35.0))
    rho = np.maximum(np.maximum(film, d1), d2)
    st = lbm.lbm_plug_analysis(rho, MID)
    drops, dmass, wmass, intact = _reference(rho, MID)
    assert st["intact"] == 0 and not intact
    assert st["n_droplets"] == drops == 2
    assert abs(st["droplet_mass"] - dmass) < 1e-12 * dmass
    assert abs(st["wall_liquid_mass"] - wmass) < 1e-12 * wmass
    # centre row crosses the larger droplet: its ends bracket the disk
    assert 140.0 - 0.5 < st["x_rear"] < 141.0 and 159.0 < st["x_front"] < 160.5


def test_random_fields_match_labelling(lbm):
    rng = np.random.default_rng(4)
    for _ in range(5):
        rho = RG + (RL - RG) * (rng.random((40, 70)) > 0.55)
        st = lbm.lbm_plug_analysis(rho, MID)
        drops, dmass, wmass, intact = _reference(rho, MID)
        assert st["n_droplets"] == drops and st["intact"] == int(intact)
        assert abs(st["droplet_mass"] - dmass) < 1e-12 * max(dmass, 1)


def test_gas_only_and_bad_arguments(lbm):
    st = lbm.lbm_plug_analysis(np.full((20, 30), RG), MID)
    assert np.isnan(st["x_rear"]) and np.isnan(st["x_front"]) and st["intact"] == 0 and st["n_droplets"] == 0
    with pytest.raises(lbm.LBMError):
        lbm.lbm_plug_analysis(np.full((3, 30), RG), MID)

"""Plug rupture and the wall-load trends of the parameter study (Sec. 3.3, Figs. 10-12).

- The trend quantities (wall-load extrema over a window of steps after the
  diagnostics restart, and the plug analysis of the density) from an FP64 GPU
  run equal the oracle's on a small channel under the paper's body-force drive.
- On the paper's proportions (1500 x 202 lattice, radius R = 100, film
  0.15 R, plug 1 R) the plug ruptures, and the directions the paper reports
  hold: the rupture comes earlier and the wall shear excursion grows with the
  force; the excursions grow with the plug length; a thin film (0.1 R) sees
  larger excursions than a thick one (0.2 R).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_08301_gb300 import build
    build.build()
    import paper_2103_08301_gb300 as m
    return m


def _oracle_coexistence(orc):
    """A consistent operating point from the oracle's own relaxed slab."""
    s = orc.Setup(nx=2, ny=96, T_over_Tc=0.85, kappa=0.5)
    g, l, _ = s.coexistence()
    f, _ = orc.run(s, orc.init(s, synth.slab_rho0(2, 96, 24, 72, l, g, width=4)), 15000)
    r = orc.fields(s, f)["rho"][:, 0]
    return r[0], r[48], orc.cs_p0(s.a, s.b, s.R, s.T, r[0])


def test_trend_quantities_match_the_oracle(orc, lbm):
    from paper_2103_08301_gb300 import trends
    nx, ny, film, plug, G = 240, 34, 4, 24, 2e-6
    settle, steps = 200, 800
    coex = _oracle_coexistence(orc)
    got = trends.rupture_run(nx, ny, film, plug, G, plug_x=48, precision=64, coex=coex, settle=settle,
                             every=steps, window=0, max_steps=settle + steps)
    rg, rl, ps = coex
    s = orc.Setup(nx=nx, ny=ny, walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5, dp=0.0, p_ref=ps, gx=G)
    f = orc.init(s, synth.airway_rho0(nx, ny, film, 48, plug, rl, rg))
    f, _ = orc.run(s, f, settle)
    f, d = orc.run(s, f, steps)
    assert abs(got["dP_wall"] - (d["pw_max"] - d["pw_min"])) <= 1e-10 * (d["pw_max"] - d["pw_min"])
    assert abs(got["dtau_wall"] - (d["tw_max"] - d["tw_min"])) <= 1e-9 * (d["tw_max"] - d["tw_min"])
    st = lbm.lbm_plug_analysis(orc.fields(s, f)["rho"], 0.5 * (rg + rl))
    last = got["history"][-1]
    assert last[0] == settle + steps
    assert abs(last[1] - st["x_rear"]) < 1e-8 and abs(last[2] - st["x_front"]) < 1e-8
    assert last[3] == st["intact"] and last[4] == st["n_droplets"]


def test_rupture_trends_on_the_paper_proportions(lbm):
    from paper_2103_08301_gb300 import trends
    base = dict(nx=1500, ny=202, film=15, plug_len=100, force=5e-7)
    rows = trends.sweep(base, {"force": [4e-7, 6e-7, 8e-7], "plug_len": [60, 100], "film": [10, 20]},
                        max_steps=60000, every=250, window=1500, settle=1000, plug_x=200)
    res = {(n, v): r for n, v, r in rows}
    for r in res.values():
        assert r["rupture_step"] is not None and not r["nan"]
    f = [res[("force", v)] for v in (4e-7, 6e-7, 8e-7)]
    assert f[0]["rupture_step"] > f[1]["rupture_step"] > f[2]["rupture_step"]
    assert f[0]["dtau_wall"] < f[1]["dtau_wall"] < f[2]["dtau_wall"]
    p60, p100 = res[("plug_len", 60)], res[("plug_len", 100)]
    assert p60["rupture_step"] < p100["rupture_step"]
    assert p60["dtau_wall"] < p100["dtau_wall"] and p60["dP_wall"] < p100["dP_wall"]
    h10, h20 = res[("film", 10)], res[("film", 20)]
    assert h10["dtau_wall"] > h20["dtau_wall"] and h10["dP_wall"] > h20["dP_wall"]

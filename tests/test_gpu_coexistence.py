"""The method's own coexistence on the GPU, and the airway at that operating point.

lbm_relaxed_coexistence relaxes a flat slab on the GPU; its bulk densities
must be the oracle's for the same slab (1e-10 in FP64), and its two bulk
pressures must agree (equal mechanical pressure across a flat interface).
With the inlet column at that pressure (p_ref = p* - dp/2) and the method's
densities as the initial state, the 512 x 128 airway keeps its gas core; with
the Maxwell reference (the default) its inlet vapour is supersaturated and the
channel floods.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("precision,tol", [(64, 1e-10), (32, 2e-5)])
def test_relaxed_coexistence_matches_the_oracle_slab(orc, lbm, precision, tol):
    ny, steps = 192, 20000
    eos = lbm.lbm_eos(1.0, 4.0, 1.0, 0.85, 1.0, 0.5)
    got = lbm.lbm_relaxed_coexistence(eos, 1.0, None, precision, ny, steps)
    s = orc.Setup(nx=2, ny=ny, T_over_Tc=0.85, kappa=0.5)
    g, l, _ = s.coexistence()
    y = np.arange(ny, dtype=np.float64)
    sl = 0.5 * (np.tanh(2 * (y - 0.25 * ny) / 4.0) - np.tanh(2 * (y - 0.75 * ny) / 4.0))
    f, _ = orc.run(s, orc.init(s, np.tile((g + (l - g) * sl)[:, None], (1, 2))), steps)
    r = orc.fields(s, f)["rho"][:, 0]
    assert abs(got["rho_g"] / r[0] - 1) <= tol
    assert abs(got["rho_l"] / r[ny // 2] - 1) <= tol
    # equal bulk pressures once settled (exact at convergence, pinned on the
    # oracle after 40000 steps; 20000 steps leave ~2e-4)
    assert abs(got["p_gas"] / got["p_liq"] - 1) <= 1e-3
    assert got["rho_g"] < 0.75 * g  # the method's vapour, well below Maxwell's at this width


def test_airway_at_the_method_coexistence_keeps_its_gas_core(lbm):
    nx, ny, dp = 512, 128, 1e-3
    eos = lbm.lbm_eos(1.0, 4.0, 1.0, 0.85, 1.0, 0.5)
    c = lbm.lbm_relaxed_coexistence(eos, 1.0, None, 64, 192, 40000)
    rho0 = lbm.lbm_airway_rho0(nx, ny, 6, 128, 48, c["rho_l"], c["rho_g"])
    mid = 0.5 * (c["rho_g"] + c["rho_l"])
    frac = {}
    for name, p_ref in (("maxwell", None), ("method", c["p_gas"] - 0.5 * dp)):
        with lbm.Lattice(nx, ny, rho0, walls=True, bc_x=True, precision=32, T_over_Tc=0.85, kappa=0.5, dp=dp,
                         p_ref=p_ref) as lat:
            lat.step(4000)
            r = lat.fields()["rho"].astype(np.float64)
        frac[name] = float((r[ny // 2 - 10:ny // 2 + 10, 8:100] > mid).mean())
        if name == "method":
            st = lbm.lbm_plug_analysis(r, mid)
            assert st["intact"] == 1  # the plug still closes the channel
    assert frac["maxwell"] > 0.5 and frac["method"] == 0.0, frac


@pytest.mark.parametrize("precision", [32, 64])
def test_gpu_slab_meets_maxwell_at_the_cancelling_relaxation_time(orc, lbm, precision):
    """The GPU step's own flat interface at tau = 1.36, 0.85 Tc: both bulk
    densities within 1% of the Maxwell construction (the oracle's, pinned to
    scipy's equal-area solution)."""
    eos = lbm.lbm_eos(1.0, 4.0, 1.0, 0.85, 1.0, 0.5)
    got = lbm.lbm_relaxed_coexistence(eos, 1.36, None, precision, 192, 60000)
    g, l, _ = orc.Setup(nx=2, ny=2, T_over_Tc=0.85, kappa=0.5).coexistence()
    assert abs(got["rho_g"] / g - 1) < 0.01 and abs(got["rho_l"] / l - 1) < 0.01, got

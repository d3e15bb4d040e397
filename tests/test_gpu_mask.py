"""GPU parity of the general-geometry step (a per-node wall mask) through the C ABI.

- The general kernels run on a plain channel (forced with LBM_OPT_GENERAL)
  do the channel kernels' arithmetic: populations and fields bit for bit.
- Masked geometries (a constriction between pressure columns, a disk obstacle
  with a wetting offset, a cross obstacle under a body force) against the FP64
  oracle after 1000 steps: rho within 1e-4 (FP32) and 1e-11 (FP64), relative
  L-infinity, as for the channel cases.
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


CHANNELS = {
    "airway512x128": (512, 128, dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5, dp=1e-3)),
    "wet96x40": (96, 40, dict(walls=True, T_over_Tc=0.8, kappa=0.5, wet=0.01)),
    "ragged129x20": (129, 20, dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5, dp=2e-4)),
    "droplet128": (128, 128, dict(T_over_Tc=0.8, kappa=0.5)),
    "mrt_airway256x64": (256, 64, dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5, tau=1.2, dp=1e-3,
                                       collision="mrt", s_e=1 / 1.2, s_eps=1.54, s_q=1 / 1.2, s_j=1 / 1.2)),
    "tiny5x4": (5, 4, dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5, dp=1e-4)),
}


def _lat_kw(kw):
    out = dict(kw)
    if "wet" in out:
        out["wetting"] = out.pop("wet")
    return out


def _channel_rho0(orc, nx, ny, kw, seed):
    g, l, _ = orc.Setup(nx=nx, ny=ny, **kw).coexistence()
    if kw.get("walls"):
        return synth.airway_rho0(nx, ny, max(1, ny // 16), nx // 4, max(2, nx // 8), l, g, noise=1e-3, seed=seed)
    return synth.disk_rho0(nx, ny, nx // 4, l, g, noise=1e-3, seed=seed)


@pytest.mark.parametrize("name", list(CHANNELS))
@pytest.mark.parametrize("precision", [32, 64])
def test_general_kernels_match_channel_kernels_bitwise(orc, lbm, name, precision):
    nx, ny, kw = CHANNELS[name]
    rho0 = _channel_rho0(orc, nx, ny, kw, 5)
    out = []
    for general in (1, 0):
        with lbm.Lattice(nx, ny, rho0, precision=precision, **_lat_kw(kw)) as lat:
            lat.set_option(lbm.LBM_OPT_GENERAL, general)
            lat.step(150)
            out.append((lat.populations(), lat.fields(), lat.diag()))
    u = np.uint32 if precision == 32 else np.uint64
    assert np.array_equal(out[0][0].view(u), out[1][0].view(u))
    for k in ("rho", "vx", "vy", "tau_wall", "p_wall"):
        assert np.array_equal(out[0][1][k].view(u), out[1][1][k].view(u)), k
    d0, d1 = out[0][2], out[1][2]
    for k in ("tau_wall_min", "tau_wall_max", "p_wall_min", "p_wall_max", "nan_detected"):
        assert d0[k] == d1[k], k
    # the sums reduce in another order
    assert abs(d0["mass"] / d1["mass"] - 1) <= (1e-13 if precision == 64 else 1e-6)
    assert abs(d0["wall_shear_sum"] - d1["wall_shear_sum"]) <= 1e-6 * abs(d1["wall_shear_sum"]) + 1e-12


def _constriction(nx, ny):
    m = np.zeros((ny, nx), np.uint8)
    m[1:ny // 4, nx // 2 - 12:nx // 2 + 12] = 1
    m[ny - ny // 4:ny - 1, nx // 2 - 12:nx // 2 + 12] = 1
    return m


def _disk(nx, ny):
    yy, xx = np.mgrid[0:ny, 0:nx]
    return ((xx - 0.6 * nx) ** 2 + (yy - 0.5 * ny) ** 2 <= 100).astype(np.uint8)


def _cross(nx, ny):
    m = np.zeros((ny, nx), np.uint8)
    c, r = ny // 2, ny // 2 - 1
    m[c - 6:c + 6, nx // 2 - 2:nx // 2 + 2] = 1
    m[c - 2:c + 2, nx // 2 - 8:nx // 2 + 8] = 1
    return m


MASKED = {
    # a constriction (blocks on both walls) between pressure columns, two-phase airway
    "constriction256x64": (256, 64, _constriction, dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5, dp=1e-3)),
    # a disk obstacle in a periodic box with a droplet next to it and a wetting offset
    "disk128x96": (128, 96, _disk, dict(T_over_Tc=0.8, kappa=0.5, wet=0.005)),
    # a cross obstacle in a walled channel under a body force (diagonal ghost rule)
    "cross160x48": (160, 48, _cross, dict(walls=True, T_over_Tc=0.8, kappa=0.5, gx=2e-6, wet=0.003)),
}


def _masked_rho0(orc, name, nx, ny, kw):
    g, l, _ = orc.Setup(nx=nx, ny=ny, **kw).coexistence()
    if name.startswith("constriction"):
        return synth.airway_rho0(nx, ny, 5, 40, 30, l, g, noise=1e-3, seed=2)
    if name.startswith("disk"):
        return synth.disk_rho0(nx, ny, 14, l, g, noise=1e-3, seed=3, centre=(0.35 * nx, 0.5 * ny))
    return synth.airway_rho0(nx, ny, 4, 100, 12, l, g, noise=1e-3, seed=4)


@pytest.mark.parametrize("name", list(MASKED))
@pytest.mark.parametrize("precision,tol", [(64, 1e-11), (32, 1e-4)])
def test_masked_geometry_parity_after_1000_steps(orc, lbm, name, precision, tol):
    nx, ny, make, kw = MASKED[name]
    mask = make(nx, ny)
    rho0 = _masked_rho0(orc, name, nx, ny, kw)
    s = orc.Setup(nx=nx, ny=ny, mask=mask, **kw)
    f_ref, d_ref = orc.run(s, orc.init(s, rho0), 1000)
    ref = orc.fields(s, f_ref)
    with lbm.Lattice(nx, ny, rho0, precision=precision, mask=mask, **_lat_kw(kw)) as lat:
        assert lat.launch_info()["threads"] == 256  # the general-geometry kernels run
        lat.step(1000)
        got = lat.fields()
        d = lat.diag()
    err = np.abs(got["rho"] - ref["rho"]).max() / np.abs(ref["rho"]).max()
    assert err <= tol, f"{name} fp{precision}: rel Linf(rho) {err:.3e}"
    assert (got["rho"][mask == 1] == 0).all()
    vscale = max(np.abs(ref["vx"]).max(), np.abs(ref["vy"]).max(), 1e-12)
    verr = max(np.abs(got["vx"] - ref["vx"]).max(), np.abs(got["vy"] - ref["vy"]).max()) / vscale
    assert verr <= (1e-9 if precision == 64 else 3e-2), f"velocity {verr:.3e}"
    assert abs(d["mass"] / d_ref["mass"] - 1) <= (1e-12 if precision == 64 else 1e-5)
    if s.walls:
        J = d_ref["J"]
        Jscale = max(abs(J), 1000 * 2 * nx * max(abs(d_ref["tw_min"]), abs(d_ref["tw_max"])) * 1e-3)
        assert abs(d["wall_shear_sum"] - J) <= (1e-9 if precision == 64 else 1e-2) * Jscale
        tw_scale = max(np.abs(ref["tau_wall"]).max(), 1e-12)
        assert np.abs(got["tau_wall"] - ref["tau_wall"]).max() <= (1e-9 if precision == 64 else 3e-2) * tw_scale
        pw_scale = np.abs(ref["p_wall"]).max()
        assert np.abs(got["p_wall"] - ref["p_wall"]).max() <= (1e-12 if precision == 64 else 1e-3) * pw_scale


def test_mask_single_step_every_population(orc, lbm):
    """One FP64 step from a random state around the cross obstacle: every
    population matches the oracle (bounce-back slots included)."""
    nx, ny = 64, 40
    mask = _cross(nx, ny)
    kw = dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5, dp=5e-4, wet=0.002)
    s = orc.Setup(nx=nx, ny=ny, mask=mask, **kw)
    g, l, _ = s.coexistence()
    rng = np.random.default_rng(21)
    rho0 = g + (l - g) * rng.random((ny, nx))
    f0 = orc.init(s, rho0) * (1 + 0.05 * rng.standard_normal((9, ny, nx)))
    f1, _ = orc.step(s, f0)
    with lbm.Lattice(nx, ny, rho0, precision=64, mask=mask, **_lat_kw(kw)) as lat:
        lat.load_populations(f0)
        lat.step(1)
        got = lat.populations()
    assert np.abs(got - f1).max() <= 1e-14 * np.abs(f1).max()


def test_mask_argument_checks(lbm):
    nx, ny = 64, 16
    rho0 = np.full((ny, nx), 0.1)
    bad = np.zeros((ny, nx), np.uint8)
    bad[5, 1] = 1  # next to the inlet column
    with pytest.raises(lbm.LBMError) as ei:
        lbm.Lattice(nx, ny, rho0, walls=True, bc_x=True, dp=1e-4, T_over_Tc=0.85, mask=bad)
    assert ei.value.status == lbm.LBM_ERR_ARG
    # a mask that marks only the wall rows keeps the channel kernels
    walls_only = np.zeros((ny, nx), np.uint8)
    walls_only[0] = walls_only[-1] = 1
    with lbm.Lattice(nx, ny, rho0, walls=True, T_over_Tc=0.85, mask=walls_only) as lat:
        assert lat.launch_info()["threads"] != 256 or lat.launch_info()["staged"]

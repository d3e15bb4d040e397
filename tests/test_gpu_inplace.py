"""In-place streaming contexts (lbm_init_inplace: one population array, the AA
pattern) against two-array contexts and the FP64 oracle.

The in-place step runs the same node arithmetic as the two-array kernels, so
populations and fields agree bit for bit; the diagnostic sums are summed in
another order and agree to rounding. Slots that no population reaches (wall
rows, the directions entering a pressure column from outside) hold different
stale values in the two layouts and are not compared.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from test_gpu_parity import CASES, _lat_kw, _rho0

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


def _fluid(ny, nx, kw):
    m = np.ones((ny, nx), bool)
    if kw.get("walls"):
        m[0, :] = m[-1, :] = False
    if kw.get("bc_x"):
        m[:, 0] = m[:, -1] = False
    return m


def _same_bits(a, b):
    u = np.uint64 if a.dtype == np.float64 else np.uint32
    return np.array_equal(a.view(u), b.view(u))


def _check_diag(da, db, precision):
    for k in ("tau_wall_min", "tau_wall_max", "p_wall_min", "p_wall_max", "nan_detected", "step"):
        assert da[k] == db[k], k
    # the two-array FP32 kernels add up to 16 rows per lane in FP32 before
    # their compensated sum (relative error up to 16 x 2^-24 = 1e-6); the
    # in-place kernel compensates every addition
    assert abs(da["mass"] / db["mass"] - 1) <= (1e-12 if precision == 64 else 1e-6)
    assert abs(da["wall_shear_sum"] - db["wall_shear_sum"]) <= 1e-9 * max(1.0, abs(db["wall_shear_sum"]))


NAMES = ["droplet128", "airway512x128", "ragged200x37", "ragged129x20", "wet96x40", "pr_droplet96",
         "mrt_pr_droplet96", "mrt_airway256x64", "bodyforce256x64"]


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", [32, 64])
def test_inplace_matches_two_array_context_bitwise(orc, lbm, name, precision):
    """101 steps (the array ends in the odd-parity layout), the fields and
    populations read back through the layout swap, then 60 more from the
    natural layout: identical to a two-array context throughout."""
    c = CASES[name]
    nx, ny, kw = c["nx"], c["ny"], c["kw"]
    rho0 = _rho0(orc, name, c)
    out = []
    for inplace in (False, True):
        with lbm.Lattice(nx, ny, rho0, precision=precision, inplace=inplace, **_lat_kw(kw)) as lat:
            rec = []
            for n in (101, 60):
                lat.step(n)
                rec.append((lat.fields(), lat.populations(), lat.diag()))
            out.append(rec)
    m = _fluid(ny, nx, kw)
    for (fa, pa, da), (fb, pb, db) in zip(*out):
        assert _same_bits(pa[:, m], pb[:, m])
        for k in ("rho", "vx", "vy", "tau_wall", "p_wall"):
            assert _same_bits(fa[k], fb[k]), k
        _check_diag(da, db, precision)


@pytest.mark.parametrize("nx,ny,walls,bc_x", [(4, 4, True, True), (5, 4, True, False), (1, 9, False, False),
                                              (7, 3, False, False), (33, 35, True, True), (32, 11, True, True),
                                              (65, 19, True, True), (40, 12, False, True), (130, 5, True, True)])
@pytest.mark.parametrize("precision", [64, 32])
def test_inplace_tiny_and_tile_edge_grids_against_oracle(orc, lbm, nx, ny, walls, bc_x, precision):
    """Grids smaller than one 32 x 8 tile (periodic axes wrap several times
    within a tile's halo), grids whose outlet column would open a tile
    (nx - 1 a multiple of 32: the tiles shift by one column) and whose
    wall-shear rows ny-3 | ny-2 would fall in two tiles ((ny - 3) a multiple of
    8: the tiles shift by one row), over an odd number of steps: populations of
    the fluid nodes against the oracle, and bit for bit against a two-array
    context."""
    kw = dict(walls=walls, bc_x=bc_x, T_over_Tc=0.85, kappa=0.5, dp=1e-4 if bc_x else 0.0)
    s = orc.Setup(nx=nx, ny=ny, **kw)
    g, l, _ = s.coexistence()
    rng = np.random.default_rng(nx * 100 + ny + 3)
    rho0 = g + (l - g) * rng.random((ny, nx)) * 0.3
    steps = 201
    f_ref, d_ref = orc.run(s, orc.init(s, rho0), steps)
    out = []
    for inplace in (True, False):
        with lbm.Lattice(nx, ny, rho0, precision=precision, inplace=inplace, **kw) as lat:
            lat.step(steps)
            out.append((lat.populations(), lat.fields(), lat.diag()))
    m = _fluid(ny, nx, kw)
    (pa, fa, da), (pb, fb, db) = out
    if precision == 64:
        assert np.abs(pa[:, m] - f_ref[:, m]).max() <= 1e-12
    else:
        ref = orc.fields(s, f_ref)["rho"]
        assert np.abs(fa["rho"].astype(np.float64) - ref).max() <= 1e-4 * np.abs(ref).max()
    assert abs(da["mass"] - d_ref["mass"]) <= (1e-12 if precision == 64 else 1e-5) * d_ref["mass"]
    if walls:
        tw = max(abs(d_ref["tw_min"]), abs(d_ref["tw_max"]))
        for d in (da, db):
            assert abs(d["wall_shear_sum"] - d_ref["J"]) <= (1e-9 if precision == 64 else 3e-5) * max(
                abs(d_ref["J"]), steps * 2 * nx * tw * 1e-3)
    assert _same_bits(pa[:, m], pb[:, m])
    for k in ("rho", "vx", "vy", "tau_wall", "p_wall"):
        assert _same_bits(fa[k], fb[k]), k
    _check_diag(da, db, precision)


def test_inplace_graph_replay_and_checkpoint(orc, lbm):
    """On a context with a stream of its own, lbm_step replays graphs of 64
    steps from the natural layout (a run that starts from the odd-parity
    layout takes one single step first): identical to single launches. A
    checkpoint taken in the odd-parity layout restores and resumes bit for
    bit, and does not restore into a two-array context."""
    import torch
    c = CASES["airway512x128"]
    nx, ny, kw = c["nx"], c["ny"], _lat_kw(c["kw"])
    rho0 = _rho0(orc, "airway512x128", c)
    pops = []
    for graph in (64, 0):
        st = torch.cuda.Stream()
        with lbm.Lattice(nx, ny, rho0, precision=32, inplace=True, stream=st, **kw) as lat:
            lat.set_option(lbm.LBM_OPT_GRAPH_STEPS, graph)
            lat.step(1)
            lat.step(130)
            lat.step(64)
            pops.append(lat.populations())
    m = _fluid(ny, nx, c["kw"])
    assert _same_bits(pops[0][:, m], pops[1][:, m])

    with lbm.Lattice(nx, ny, rho0, precision=32, inplace=True, **kw) as lat:
        lat.step(51)
        ck = lat.checkpoint()
        lat.step(30)
        a = lat.populations()
        da = lat.diag()
        lat.restore(ck)
        lat.step(30)
        b = lat.populations()
        db = lat.diag()
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
        assert da == db
    with lbm.Lattice(nx, ny, rho0, precision=32, **kw) as two:
        assert len(ck) < two.checkpoint().size
        with pytest.raises(lbm.LBMError) as ei:
            two.restore(np.concatenate([ck, np.zeros(two.checkpoint().size - len(ck), np.uint8)]))
        assert ei.value.status == lbm.LBM_ERR_STATE


def test_inplace_storage_and_options(orc, lbm):
    """An in-place context steps in a caller's workspace of
    lbm_workspace_bytes_inplace bytes, reports its tile grid, and rejects the
    options it has no kernels for."""
    import torch
    c = CASES["airway512x128"]
    kw = _lat_kw(c["kw"])
    rho0 = _rho0(orc, "airway512x128", c)
    ws = torch.empty(lbm.lbm_workspace_bytes_inplace(lbm.lbm_grid(512, 128, 1, 1, 32)), dtype=torch.uint8,
                     device="cuda")
    with lbm.Lattice(512, 128, rho0, precision=32, inplace=True, workspace=ws, **kw) as lat:
        info = lat.launch_info()
        assert info["threads"] == 128 and info["units"] == 16 * 16 and not info["staged"]  # FP32: row pairs
        for opt in (lbm.LBM_OPT_GENERAL, lbm.LBM_OPT_FAULT_SKIP_COPY):
            with pytest.raises(lbm.LBMError) as ei:
                lat.set_option(opt, 1)
            assert ei.value.status == lbm.LBM_ERR_ARG
        lat.step(10)
        assert not lat.diag()["nan_detected"]
    with pytest.raises(ValueError):
        lbm.Lattice(512, 128, rho0, precision=32, inplace=True, mask=np.zeros((128, 512)), **kw)


def test_inplace_full_size_and_64_bit_offsets(orc, lbm):
    """The benchmark channel (16384 x 2048) and a grid past 2^31 population
    slots (16384 x 14600, 64-bit offsets): an odd number of in-place steps
    against the two-array context, populations of the fluid nodes compared on
    the device bit for bit."""
    import torch
    s = orc.Setup(nx=8, ny=8, T_over_Tc=0.85, kappa=0.5)
    g, l, _ = s.coexistence()
    kw = dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5, dp=1e-3)
    for nx, ny, steps in ((16384, 2048, 21), (16384, 14600, 3)):
        rho0 = synth.airway_rho0(nx, ny, 64, 4096, 1024, l, g, noise=1e-3, seed=3)
        got = []
        for inplace in (False, True):
            with lbm.Lattice(nx, ny, rho0, precision=32, inplace=inplace, **kw) as lat:
                lat.step(steps)
                f = torch.empty((9, ny, nx), dtype=torch.float32, device="cuda")
                assert lbm.lib().lbm_populations(lat.ctx, C.c_void_p(f.data_ptr())) == lbm.LBM_OK
                torch.cuda.synchronize()
                assert not lat.diag()["nan_detected"]
                got.append(f[:, 1:ny - 1, 1:nx - 1].contiguous().view(torch.int32))
                del f
        assert torch.equal(got[0], got[1]), (nx, ny)
        del got, rho0
        torch.cuda.empty_cache()

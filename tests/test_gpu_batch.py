"""Batched channels (lbm_batch_*) against single-channel contexts.

Each channel of a batch runs the same per-segment code as a single-channel
context, so its populations must agree bit for bit; per-channel diagnostics are
sums over differently cut segments and agree to rounding.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

KW = dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5)


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_08301_gb300 import build
    build.build()
    import paper_2103_08301_gb300 as m
    return m


def _channels(orc, specs):
    s = orc.Setup(nx=64, ny=16, **KW, dp=0.0)
    g, l, _ = s.coexistence()
    out = []
    for nx, ny, dp, film, plug_x, plug_len in specs:
        out.append({"nx": nx, "ny": ny, "dp": dp,
                    "rho0": synth.airway_rho0(nx, ny, film, plug_x, plug_len, l, g)})
    return out


STAGED_SPECS = [(256, 40, 1e-3, 4, 60, 30), (384, 64, 5e-4, 6, 90, 48), (1024, 96, 2e-3, 8, 256, 64),
                (132, 24, 1.5e-3, 3, 30, 20), (512, 130, 8e-4, 10, 128, 40)]
RAGGED_SPECS = [(301, 40, 1e-3, 4, 60, 30), (129, 33, 5e-4, 3, 40, 16), (250, 64, 2e-3, 6, 64, 32)]


def _single(lbm, ch, precision, steps):
    with lbm.Lattice(ch["nx"], ch["ny"], ch["rho0"], precision=precision, dp=ch["dp"], **KW) as lat:
        lat.step(steps)
        return lat.populations(), lat.diag()


@pytest.mark.parametrize("specs,staged", [(STAGED_SPECS, True), (RAGGED_SPECS, True), (RAGGED_SPECS, False)])
@pytest.mark.parametrize("precision", [32, 64])
def test_batch_matches_single_channels_bitwise(orc, lbm, specs, staged, precision):
    # ragged widths are staged through padded row pitches; the register-
    # prefetch kernel is forced with the staging option
    chans = _channels(orc, specs)
    steps = 150  # two 64-step graph replays and 22 single launches
    with lbm.Batch(chans, precision=precision, **KW) as b:
        if not staged:
            b.set_option(lbm.LBM_OPT_STAGED, 0)
        assert b.launch_info()["staged"] == int(staged)
        b.step(steps)
        got = [(b.populations(c), b.diag(c)) for c in range(len(chans))]
    u = np.uint32 if precision == 32 else np.uint64
    for c, ch in enumerate(chans):
        f_ref, d_ref = _single(lbm, ch, precision, steps)
        assert np.array_equal(got[c][0].view(u), f_ref.view(u)), f"channel {c}"
        d = got[c][1]
        assert d["step"] == steps
        assert abs(d["mass"] / d_ref["mass"] - 1) < (1e-13 if precision == 64 else 1e-6)
        assert abs(d["wall_shear_sum"] - d_ref["wall_shear_sum"]) <= 1e-9 * abs(d_ref["wall_shear_sum"]) + 1e-15
        assert d["tau_wall_max"] == pytest.approx(d_ref["tau_wall_max"], rel=1e-6, abs=1e-12)
        assert d["rho_in"] == d_ref["rho_in"] and d["rho_out"] == d_ref["rho_out"]


def test_batch_matches_oracle_fp64(orc, lbm):
    chans = _channels(orc, STAGED_SPECS[:3])
    with lbm.Batch(chans, precision=64, **KW) as b:
        b.step(300)
        rho = [b.fields(c)["rho"] for c in range(3)]
    for c, ch in enumerate(chans):
        s = orc.Setup(nx=ch["nx"], ny=ch["ny"], dp=ch["dp"], **KW)
        f, _ = orc.run(s, orc.init(s, ch["rho0"]), 300)
        ref = orc.fields(s, f)["rho"]
        assert np.abs(rho[c] - ref).max() <= 1e-11 * np.abs(ref).max()


def test_graph_reverse_and_autotune_keep_results(orc, lbm):
    chans = _channels(orc, STAGED_SPECS)
    outs = []
    for mode in ("graph", "nograph", "reverse", "autotune"):
        with lbm.Batch(chans, precision=32, **KW) as b:
            if mode == "nograph":
                b.set_option(lbm.LBM_OPT_GRAPH_STEPS, 0)
            if mode == "reverse":
                b.set_option(lbm.LBM_OPT_REVERSE, 1)
            if mode == "autotune":
                best = b.autotune(trial_steps=4)
                assert best["ctas_per_sm"] >= 1 and best["strip"] in (64, 128)
                assert best["ms_per_step"] > 0
            b.step(130)
            outs.append(np.concatenate([b.populations(c).ravel() for c in range(len(chans))]))
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32))


def test_batch_mrt_matches_single_channels_bitwise(orc, lbm):
    # MRT collision (Eq. 2.1) set on the batch after it was built (the CUDA
    # graph is re-captured with the new arguments)
    chans = _channels(orc, STAGED_SPECS[:3])
    rates = dict(s_e=1 / 1.2, s_eps=1.54, s_j=1 / 1.2, s_q=1 / 1.2, s_nu=None)
    coll = lbm.lbm_collision(lbm.LBM_COLL_MRT, rates["s_e"], rates["s_eps"], rates["s_j"], rates["s_q"], 0.0)
    with lbm.Batch(chans, precision=32, tau=1.2, **KW) as b:
        b.step(70)  # BGK steps, graph captured
        b.set_collision(coll)
        b.step(80)
        got = [b.populations(c) for c in range(len(chans))]
    for c, ch in enumerate(chans):
        with lbm.Lattice(ch["nx"], ch["ny"], ch["rho0"], precision=32, dp=ch["dp"], tau=1.2, **KW) as lat:
            lat.step(70)
            lat.set_collision(coll)
            lat.step(80)
            ref = lat.populations()
        assert np.array_equal(got[c].view(np.uint32), ref.view(np.uint32)), f"channel {c}"


PERIODIC_SPECS = [(256, 40, 0.0, 4, 60, 30), (132, 24, 0.0, 3, 30, 20), (512, 66, 0.0, 6, 128, 40)]


@pytest.mark.parametrize("specs,kw", [(STAGED_SPECS, KW), (RAGGED_SPECS, KW),
                                      (PERIODIC_SPECS, dict(walls=True, bc_x=False, T_over_Tc=0.85, kappa=0.5))])
def test_batch_row_pair_kernel_matches_one_row_kernel(orc, lbm, specs, kw):
    """The batch's row-pair step (FP32) against its one-row step: populations
    bit for bit and per-channel diagnostic sums to rounding, with pressure columns (ragged
    widths through padded pitches) and with periodic x (wrapped halo copies)."""
    chans = _channels(orc, specs)
    for ch in chans:
        ch["gx"] = 2e-6 if not kw["bc_x"] else 0.0
    outs = []
    for rows2 in (1, 0):
        with lbm.Batch(chans, precision=32, **kw) as b:
            b.set_option(lbm.LBM_OPT_ROWS2, rows2)
            # the same strips and CTA count, hence the same segment list and
            # diagnostics order (row pairs take strips of at most 124 columns)
            b.set_option(lbm.LBM_OPT_STRIP, 124)
            b.set_option(lbm.LBM_OPT_CTAS_PER_SM, 4)
            b.step(130)
            outs.append([(b.populations(c), b.diag(c)) for c in range(len(chans))])
    for c in range(len(chans)):
        assert np.array_equal(outs[0][c][0].view(np.uint32), outs[1][c][0].view(np.uint32)), f"channel {c}"
        for k in ("tau_wall_max", "tau_wall_min"):
            assert outs[0][c][1][k] == outs[1][c][1][k], (c, k)
        # summed in another lane order
        m0, m1 = outs[0][c][1]["mass"], outs[1][c][1]["mass"]
        assert abs(m0 - m1) <= 1e-12 * m1, c
        j0, j1 = outs[0][c][1]["wall_shear_sum"], outs[1][c][1]["wall_shear_sum"]
        assert abs(j0 - j1) <= 1e-9 * abs(j1) + 1e-15, c


@pytest.mark.parametrize("specs,kw", [(RAGGED_SPECS, KW),
                                      (PERIODIC_SPECS, dict(walls=True, bc_x=False, T_over_Tc=0.85, kappa=0.5))])
def test_batch_tensor_map_stage_matches_bulk_copies(orc, lbm, specs, kw):
    """The batch's row-pair stage through per-channel tensor maps and through
    plane copies: populations and diagnostics bit for bit (same kernel body,
    same work list)."""
    chans = _channels(orc, specs)
    for ch in chans:
        ch["gx"] = 2e-6 if not kw["bc_x"] else 0.0
    outs = []
    for tma in (1, 0):
        with lbm.Batch(chans, precision=32, **kw) as b:
            b.set_option(lbm.LBM_OPT_TMA, tma)
            b.step(130)
            outs.append([(b.populations(c), b.diag(c)) for c in range(len(chans))])
    for c in range(len(chans)):
        assert np.array_equal(outs[0][c][0].view(np.uint32), outs[1][c][0].view(np.uint32)), f"channel {c}"
        assert outs[0][c][1]["mass"] == outs[1][c][1]["mass"], c


@pytest.mark.parametrize("kind", ["airway_copies", "airway_tma", "periodic"])
def test_persistent_batch_matches_per_step_launches_bitwise(orc, lbm, kind):
    """One cooperative launch carrying many steps (segments ordered by step
    counters) against one launch per step: the same populations, bit for bit,
    and the same diagnostics, over an odd number of steps (the buffers end
    swapped) and uneven channels. Both take the balanced cut of the work
    order (LBM_OPT_BAND = 0), so the segments, and with them the partial sums,
    are the same."""
    if kind == "periodic":
        kw = dict(walls=False, bc_x=False, T_over_Tc=0.8, kappa=0.5)
        g, l, _ = orc.Setup(nx=8, ny=8, **kw).coexistence()
        chans = [{"nx": nx, "ny": ny, "rho0": synth.disk_rho0(nx, ny, r, l, g, noise=1e-3, seed=nx,
                                                              centre=(0.3 * nx, 0.6 * ny))}
                 for nx, ny, r in ((256, 64, 14), (132, 40, 9), (512, 24, 7), (128, 128, 30))]
    else:
        kw = KW
        chans = _channels(orc, STAGED_SPECS + [(2048, 300, 1e-3, 12, 512, 128)])
    steps = 137
    out = []
    for persistent in (1, 0):
        with lbm.Batch(chans, precision=32, **kw) as b:
            b.set_option(lbm.LBM_OPT_TMA, 0 if kind == "airway_copies" else 1)
            b.set_option(lbm.LBM_OPT_BAND, 0)
            b.set_option(lbm.LBM_OPT_PERSISTENT, persistent)
            b.step(steps)
            out.append([(b.populations(i), b.diag(i)) for i in range(len(chans))])
    for (pa, da), (pb, db) in zip(*out):
        assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
        for k in ("mass", "wall_shear_sum", "tau_wall_min", "tau_wall_max", "p_wall_min", "p_wall_max",
                  "nan_detected"):
            assert da[k] == db[k], k


@pytest.mark.parametrize("band", [8, 37, 64, -1])
def test_band_major_work_order_matches_strip_major_bitwise(orc, lbm, band):
    """The batch's work order cut into bands (LBM_OPT_BAND) against the
    strip-by-strip order: the same populations bit for bit, the same extrema
    and error word, and sums equal to rounding (the segments change), with the
    persistent launch (segment dependencies over bands) as well."""
    chans = _channels(orc, STAGED_SPECS + [(2048, 300, 1e-3, 12, 512, 128)])
    steps = 41
    out = []
    for band_opt, persistent in ((0, 0), (band, 0), (band, 1)):
        with lbm.Batch(chans, precision=32, **KW) as b:
            b.set_option(lbm.LBM_OPT_BAND, band_opt)
            b.set_option(lbm.LBM_OPT_PERSISTENT, persistent)
            b.step(steps)
            out.append([(b.populations(i), b.diag(i)) for i in range(len(chans))])
    for other in out[1:]:
        for (pa, da), (pb, db) in zip(out[0], other):
            assert np.array_equal(pa.view(np.uint32), pb.view(np.uint32))
            for k in ("tau_wall_min", "tau_wall_max", "p_wall_min", "p_wall_max", "nan_detected"):
                assert da[k] == db[k], k
            # per-segment partials are FP32 sums of up to 16 rows per lane
            assert abs(da["mass"] / db["mass"] - 1) <= 1e-6
            assert abs(da["wall_shear_sum"] - db["wall_shear_sum"]) <= 1e-5 * abs(da["wall_shear_sum"]) + 1e-9

"""The allocation-free step (lbm_step_noalloc) against the ordinary context path.

lbm_step_noalloc serves callers that cannot call cudaMalloc when they step the
lattice (code inside a framework that owns the memory pool, a host that sizes
all buffers up front): it steps between two caller-owned buffers and keeps its
per-CTA scratch in a fixed device array.
Here the test allocates the buffers itself (with torch) and checks two calls
in a row against two lbm_step calls on a context. This file is collected last
so a failure here comes after every other test has run.
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


@pytest.mark.parametrize("precision", [32, 64])
def test_noalloc_step_matches_context_step_twice(orc, lbm, precision):
    import torch
    nx, ny = 512, 96
    kw = dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5, dp=1e-3)
    s = orc.Setup(nx=nx, ny=ny, **kw)
    g, l, _ = s.coexistence()
    rho0 = synth.airway_rho0(nx, ny, 6, 160, 48, l, g)
    tdt = torch.float32 if precision == 32 else torch.float64
    with lbm.Lattice(nx, ny, rho0, precision=precision, **kw) as lat:
        lat.step(40)
        f0 = lat.populations()
        d0 = lat.diag()
        lat.step(1)
        f1, d1 = lat.populations(), lat.diag()
        lat.step(1)
        f2, d2 = lat.populations(), lat.diag()
        grid, eos, drive = lat.grid, lat.eos, lat.drive

    # the allocation-free step uses the library's row-interleaved layout f[y][i][x]
    def to_rows(f):
        return np.ascontiguousarray(f.transpose(1, 0, 2))

    def from_rows(t):
        return np.ascontiguousarray(t.cpu().numpy().transpose(1, 0, 2))

    a = torch.from_numpy(to_rows(f0)).to("cuda", tdt)
    b = a.clone()  # slots no population reaches keep the input values, as in the context
    c = a.clone()
    diag = torch.zeros(2, 7, dtype=torch.float64, device="cuda")
    err = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    st = lbm.lbm_step_noalloc(grid, eos, 1.0, 0.0, drive, a.data_ptr(), b.data_ptr(), 0,
                              diag[0].data_ptr(), None, err[0].data_ptr())
    assert st == lbm.LBM_OK, lbm.status_string(st)
    st = lbm.lbm_step_noalloc(grid, eos, 1.0, 0.0, drive, b.data_ptr(), c.data_ptr(), 0,
                              diag[1].data_ptr(), None, err[1].data_ptr())
    assert st == lbm.LBM_OK, lbm.status_string(st)
    torch.cuda.synchronize()
    assert err.tolist() == [0, 0]  # the error word: no bad density, no stage wait gave up
    u = np.uint32 if precision == 32 else np.uint64
    # same kernel, same launch geometry: identical bits
    assert np.array_equal(from_rows(b).view(u), f1.view(u))
    assert np.array_equal(from_rows(c).view(u), f2.view(u))
    dg = diag.cpu().numpy()
    tol = 1e-12 if precision == 64 else 1e-6
    # per-call diagnostics are those of the state each call read
    assert abs(dg[0, 0] / d1["mass"] - 1) <= tol and abs(dg[1, 0] / d2["mass"] - 1) <= tol
    for k, (dj, da, db) in enumerate([(dg[0, 1], d0, d1), (dg[1, 1], d1, d2)]):
        step_J = db["wall_shear_sum"] - da["wall_shear_sum"]
        assert abs(dj - step_J) <= 1e-6 * max(abs(step_J), 1e-12) + 1e-12, (k, dj, step_J)
    assert dg[0, 6] == 0 and dg[1, 6] == 0


def test_noalloc_rejects_bad_requests(lbm):
    import torch
    g = lbm.lbm_grid(64, 32, 1, 0, 32)
    e = lbm.lbm_eos(1.0, 4.0, 1.0, 0.8, 1.0, 0.5)
    a = torch.zeros(9 * 64 * 32, dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    assert lbm.lbm_step_noalloc(g, e, 1.0, 0.0, None, a.data_ptr(), b.data_ptr(), 4097) == lbm.LBM_ERR_ARG
    assert lbm.lbm_step_noalloc(g, e, 1.0, 0.0, None, a.data_ptr(), a.data_ptr(), 0) == lbm.LBM_ERR_ARG
    assert lbm.lbm_step_noalloc(g, e, 0.5, 0.0, None, a.data_ptr(), b.data_ptr(), 0) == lbm.LBM_ERR_PARAM


@pytest.mark.parametrize("precision", [32, 64])
def test_noalloc_ragged_width_and_offset_views(orc, lbm, precision):
    """A width that is not a multiple of 4 (the context pads its rows to 304
    columns, the caller's buffers have 301) and caller buffers that start off a
    16-byte boundary (views with a one-element offset) take the register-
    prefetch kernel; both must reproduce the context step, bit for bit."""
    import torch
    nx, ny = 301, 40
    kw = dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5, dp=2e-4)
    s = orc.Setup(nx=nx, ny=ny, **kw)
    g, l, _ = s.coexistence()
    rho0 = synth.airway_rho0(nx, ny, 4, 90, 30, l, g, noise=1e-3, seed=7)
    tdt = torch.float32 if precision == 32 else torch.float64
    u = np.uint32 if precision == 32 else np.uint64
    with lbm.Lattice(nx, ny, rho0, precision=precision, **kw) as lat:
        lat.step(25)
        f0 = lat.populations()
        lat.step(1)
        f1 = lat.populations()
        lat.step(1)
        f2 = lat.populations()
        grid, eos, drive = lat.grid, lat.eos, lat.drive
    rows = np.ascontiguousarray(f0.transpose(1, 0, 2)).ravel()
    n = rows.size
    for offset in (0, 1):
        buf = torch.zeros(3 * (n + 4), dtype=tdt, device="cuda")
        views = [buf[k * (n + 4) + offset:k * (n + 4) + offset + n] for k in range(3)]
        for v in views:
            v.copy_(torch.from_numpy(rows))
        if offset:
            assert views[0].data_ptr() % 16 != 0
        err = torch.full((2,), -1, dtype=torch.int32, device="cuda")
        for k in range(2):
            st = lbm.lbm_step_noalloc(grid, eos, 1.0, 0.0, drive, views[k].data_ptr(), views[k + 1].data_ptr(),
                                      0, None, None, err[k].data_ptr())
            assert st == lbm.LBM_OK, lbm.status_string(st)
        torch.cuda.synchronize()
        assert err.tolist() == [0, 0]
        for v, ref in ((views[1], f1), (views[2], f2)):
            got = np.ascontiguousarray(v.cpu().numpy().reshape(ny, 9, nx).transpose(1, 0, 2))
            assert np.array_equal(got.view(u), ref.view(u)), offset

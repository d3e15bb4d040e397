"""Failure detection on the GPU without a GPU fault.

- A stage copy that never arrives (a test hook: the first CTA skips the copy
  of its final row pair and every wait polls a small, bounded number of
  times): the wait gives up, lbm_step reports LBM_ERR_TIMEOUT, and after
  lbm_restore the run continues bit for bit as an undisturbed one.
- A simulated allocation failure (LBM_FAULT=alloc) returns LBM_ERR_OOM and
  leaves no device memory behind.
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


@pytest.mark.parametrize("ctas_per_sm", [1, 5])
def test_lost_stage_copy_times_out_and_restore_recovers(orc, lbm, ctas_per_sm):
    import torch
    nx, ny = 512, 512
    kw = dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5, dp=1e-3)
    g, l, _ = orc.Setup(nx=nx, ny=ny, **kw).coexistence()
    rho0 = synth.airway_rho0(nx, ny, 12, 160, 48, l, g)
    with lbm.Lattice(nx, ny, rho0, precision=32, **kw) as lat:
        lat.set_option(lbm.LBM_OPT_CTAS_PER_SM, ctas_per_sm)
        assert lat.launch_info()["threads"] == 128  # the row-pair kernel
        lat.step(30)
        ck = lat.checkpoint()
        lat.step(40)
        ref, dref = lat.populations(), lat.diag()
        lat.restore(ck)
        lat.set_option(lbm.LBM_OPT_FAULT_SKIP_COPY, 1)
        assert lbm.lbm_step(lat.ctx, 1) == lbm.LBM_OK  # asynchronous: reports earlier steps
        torch.cuda.synchronize()
        assert lbm.lbm_step(lat.ctx, 0) == lbm.LBM_ERR_TIMEOUT
        assert lat.diag()["nan_detected"] == 0  # a timeout, not a bad density
        lat.set_option(lbm.LBM_OPT_FAULT_SKIP_COPY, 0)
        lat.restore(ck)
        lat.step(40)
        got, d = lat.populations(), lat.diag()
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    assert d["mass"] == dref["mass"] and d["wall_shear_sum"] == dref["wall_shear_sum"]


def test_simulated_allocation_failure_leaks_nothing(lbm, monkeypatch):
    import torch
    nx, ny = 2048, 1024
    rho0 = np.full((ny, nx), 0.1)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    monkeypatch.setenv("LBM_FAULT", "alloc")
    for _ in range(3):
        with pytest.raises(lbm.LBMError) as ei:
            lbm.Lattice(nx, ny, rho0, walls=True, T_over_Tc=0.85)
        assert ei.value.status == lbm.LBM_ERR_OOM
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < 4 << 20  # three 150 MB workspaces were allocated and released
    monkeypatch.delenv("LBM_FAULT")
    with lbm.Lattice(nx, ny, rho0, walls=True, T_over_Tc=0.85) as lat:
        lat.step(2)

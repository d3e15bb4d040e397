"""CPU tests of the C ABI: the library builds, exports every symbol that
include/lbm.h declares, validates its arguments, and its host helpers agree
with the oracle / the seeded input generators (no GPU calls)."""
import math
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lbm():
    from paper_2103_08301_gb300 import build
    build.build()
    import paper_2103_08301_gb300 as m
    m.lib()
    return m


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(lbm):
    names = _declared_symbols()
    assert len(names) >= 18
    lib = lbm.lib()
    for n in names:
        assert hasattr(lib, n), n
    # and the binding covers the same set
    assert set(names) == set(lbm._SIGS), set(names) ^ set(lbm._SIGS)


def test_status_strings(lbm):
    for s in range(8):
        assert lbm.status_string(s)
    assert "wait" in lbm.status_string(lbm.LBM_ERR_TIMEOUT)
    assert lbm.status_string(0) == "ok"


def test_workspace_bytes(lbm):
    g = lbm.lbm_grid(256, 64, 1, 1, 32)
    b32 = lbm.lbm_workspace_bytes(g)
    assert b32 >= 2 * 9 * 256 * 64 * 4
    g64 = lbm.lbm_grid(256, 64, 1, 1, 64)
    assert lbm.lbm_workspace_bytes(g64) >= 2 * 9 * 256 * 64 * 8
    for bad in [lbm.lbm_grid(0, 64, 0, 0, 32), lbm.lbm_grid(64, 3, 1, 0, 32),
                lbm.lbm_grid(3, 64, 0, 1, 32), lbm.lbm_grid(64, 64, 0, 0, 16),
                lbm.lbm_grid(64, 64, 2, 0, 32),
                lbm.lbm_grid(1 << 16, 1 << 15, 0, 0, 32),  # 2^31 nodes
                lbm.lbm_grid(1, 1 << 28, 0, 0, 32)]:       # 9 ny >= 2^31 plane-rows
        assert lbm.lbm_workspace_bytes(bad) == 0
    # past 2^31 population slots a context takes 64-bit offsets
    big = lbm.lbm_grid(16384, 16384, 1, 1, 32)
    assert lbm.lbm_workspace_bytes(big) >= 2 * 9 * 16384 * 16384 * 4


def test_inplace_workspace_bytes(lbm):
    """An in-place context stores one population array, a density plane and a
    small side buffer: 40 (FP32) or 80 (FP64) bytes per node plus alignment."""
    for prec, sz in ((32, 4), (64, 8)):
        g = lbm.lbm_grid(1024, 256, 1, 1, prec)
        one, two = lbm.lbm_workspace_bytes_inplace(g), lbm.lbm_workspace_bytes(g)
        assert 10 * sz * 1024 * 256 <= one < 10 * sz * 1024 * 256 + (1 << 20)
        assert 18 * sz * 1024 * 256 <= two and one < 0.6 * two
    assert lbm.lbm_workspace_bytes_inplace(lbm.lbm_grid(0, 64, 0, 0, 32)) == 0
    big = lbm.lbm_grid(16384, 14600, 1, 1, 32)  # 64-bit population offsets
    assert lbm.lbm_workspace_bytes_inplace(big) >= 10 * 4 * 16384 * 14600
    e = lbm.lbm_eos(1.0, 4.0, 1.0, 0.8, 1.0, 0.5)
    rho0 = np.full((16, 16), 0.1)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_init_inplace(lbm.lbm_grid(16, 16, 0, 0, 32), e, 0.5, 0.0, None, rho0)  # tau must exceed 1/2
    assert ei.value.status == lbm.LBM_ERR_PARAM
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_init_inplace(lbm.lbm_grid(0, 16, 0, 0, 32), e, 1.0, 0.0, None, rho0)
    assert ei.value.status == lbm.LBM_ERR_ARG


def test_paths_with_32_bit_offsets_reject_larger_grids(lbm):
    """The batch, the allocation-free step and the adjoint keep 9 pitch ny < 2^31
    and refuse larger grids before touching the GPU."""
    import ctypes as C
    big = lbm.lbm_grid(16384, 14600, 1, 1, 32)
    e = lbm.lbm_eos(1.0, 4.0, 1.0, 0.85, 1.0, 0.5)
    one = (C.c_double * 1)(0.1)
    rho = (C.POINTER(C.c_double) * 1)(C.cast(one, C.POINTER(C.c_double)))
    out = C.c_void_p()
    assert lbm.lib().lbm_batch_init(1, C.byref(big), C.byref(e), 1.0, 0.0, None, rho, None,
                                    C.byref(out)) == lbm.LBM_ERR_ARG
    assert lbm.lib().lbm_step_noalloc(C.byref(big), C.byref(e), 1.0, 0.0, None, C.c_void_p(16), C.c_void_p(32),
                                      0, None, None, None) == lbm.LBM_ERR_ARG
    assert lbm.lib().lbm_adjoint_init(C.byref(big), C.byref(e), 1.0, 0.0, 10, 0, None,
                                      C.byref(out)) == lbm.LBM_ERR_ARG


def test_init_rejects_bad_arguments_before_touching_the_gpu(lbm):
    g = lbm.lbm_grid(16, 16, 0, 0, 32)
    e = lbm.lbm_eos(1.0, 4.0, 1.0, 0.8, 1.0, 0.5)
    rho0 = np.full((16, 16), 0.1)
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_init(g, e, 0.5, 0.0, None, rho0)  # tau must exceed 1/2
    assert ei.value.status == lbm.LBM_ERR_PARAM
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_init(lbm.lbm_grid(0, 16, 0, 0, 32), e, 1.0, 0.0, None, rho0)
    assert ei.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_init(g, lbm.lbm_eos(1.0, 4.0, 1.0, 0.8, 0.0, 0.5), 1.0, 0.0, None, rho0)
    assert ei.value.status == lbm.LBM_ERR_PARAM
    assert lbm.lib().lbm_step(None, 1) == lbm.LBM_ERR_ARG
    lbm.lib().lbm_free(None)  # NULL-safe


@pytest.mark.parametrize("t", [0.72, 0.8, 0.85, 0.95])
def test_coexistence_helper_matches_oracle(lbm, orc, t):
    Tc, g, l, p = lbm.lbm_coexistence(lbm.lbm_eos(1.0, 4.0, 1.0, t, 1.0, 0.5))
    Tc2, _ = orc.cs_critical()
    g2, l2, p2 = orc.maxwell(1.0, 4.0, 1.0, t * Tc2)
    assert abs(Tc / Tc2 - 1) < 1e-14
    assert abs(g / g2 - 1) < 1e-11 and abs(l / l2 - 1) < 1e-12 and abs(p / p2 - 1) < 1e-11
    with pytest.raises(lbm.LBMError):
        lbm.lbm_coexistence(lbm.lbm_eos(1.0, 4.0, 1.0, 1.05, 1.0, 0.5))


def test_initial_profiles_match_seeded_generators(lbm):
    a = lbm.lbm_airway_rho0(300, 70, 8, 60, 40, 0.28, 0.03, 4.0, 1e-3, 7)
    b = synth.airway_rho0(300, 70, 8, 60, 40, 0.28, 0.03, width=4.0, noise=1e-3, seed=7)
    assert np.abs(a - b).max() < 1e-15
    c = lbm.lbm_disk_rho0(128, 96, 64.0, 48.0, 30.0, 0.3, 0.02, 4.0, 1e-3, 1)
    d = synth.disk_rho0(128, 96, 30.0, 0.3, 0.02, width=4.0, noise=1e-3, seed=1)
    assert np.abs(c - d).max() < 1e-15
    # the noise bits themselves are identical (same published generator)
    n1 = lbm.lbm_disk_rho0(64, 8, 0.0, 0.0, -10.0, 0.0, 0.0, 4.0, 1.0, 3)
    n2 = synth.node_noise(64, 8, 1.0, 3)
    assert np.array_equal(n1, n2)


def test_splitmix64_known_values():
    # Reference outputs of SplitMix64 seeded with 0 (successive states
    # k * 0x9E3779B97F4A7C15), published with the generator.
    gamma = 0x9E3779B97F4A7C15
    states = np.array([(k * gamma) % (1 << 64) for k in range(3)], dtype=np.uint64)
    out = [int(v) for v in synth.splitmix64(states)]
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_airway_tangent_matches_central_differences(lbm):
    # d rho0 / d film and d rho0 / d plug_len against central differences of
    # the seeded generator (the profile is smooth away from the film/plug tie)
    nx, ny, h, x0, L, rl, rg = 160, 48, 6.3, 40.0, 27.7, 0.28, 0.03
    d_film, d_plug = lbm.lbm_airway_rho0_tangent(nx, ny, h, x0, L, rl, rg, 4.0)
    e = 1e-5
    fd_film = (synth.airway_rho0(nx, ny, h + e, x0, L, rl, rg) - synth.airway_rho0(nx, ny, h - e, x0, L, rl, rg)) / (2 * e)
    fd_plug = (synth.airway_rho0(nx, ny, h, x0, L + e, rl, rg) - synth.airway_rho0(nx, ny, h, x0, L - e, rl, rg)) / (2 * e)
    assert np.abs(d_film - fd_film).max() < 1e-8
    assert np.abs(d_plug - fd_plug).max() < 1e-8
    assert np.abs(d_film).max() > 0.01 and np.abs(d_plug).max() > 0.01


def test_adjoint_rejects_bad_arguments_before_touching_the_gpu(lbm):
    import ctypes as C
    e = lbm.lbm_eos(1.0, 4.0, 1.0, 0.85, 1.0, 0.5)
    h = C.c_void_p()
    # the forward precision is 32 or 64
    st = lbm.lib().lbm_adjoint_init(C.byref(lbm.lbm_grid(64, 32, 1, 1, 16)), C.byref(e), 1.0, 0.0, 10, 0, None,
                                    C.byref(h))
    assert st == lbm.LBM_ERR_ARG and not h.value
    st = lbm.lib().lbm_adjoint_init(C.byref(lbm.lbm_grid(64, 32, 1, 1, 64)), C.byref(e), 1.0, 0.0, 0, 0, None,
                                    C.byref(h))
    assert st == lbm.LBM_ERR_ARG
    st = lbm.lib().lbm_adjoint_init(C.byref(lbm.lbm_grid(64, 32, 1, 1, 64)), C.byref(e), 0.5, 0.0, 10, 0, None,
                                    C.byref(h))
    assert st == lbm.LBM_ERR_PARAM
    g = (C.c_double * 3)()
    assert lbm.lib().lbm_adjoint_backward(None, 1.0, 0.0, None, g) == lbm.LBM_ERR_ARG
    assert lbm.lib().lbm_adjoint_set_precision(None, 32) == lbm.LBM_ERR_ARG
    assert lbm.lib().lbm_diag_async(None, C.c_void_p(64)) == lbm.LBM_ERR_ARG
    lbm.lib().lbm_adjoint_free(None)  # NULL-safe


def test_collision_setter_validates_before_touching_the_gpu(lbm):
    import ctypes as C
    mrt = lbm.lbm_collision(lbm.LBM_COLL_MRT, 1.64, 1.54, 1.0, 1.7, 0.0)
    assert lbm.lib().lbm_set_collision(None, C.byref(mrt)) == lbm.LBM_ERR_ARG


def test_pr_coexistence_helper_matches_oracle(lbm, orc):
    for tr in (0.5, 0.6, 0.8):
        Tc, g, l, p = lbm.lbm_coexistence(lbm.lbm_eos(2 / 49, 2 / 21, 1.0, tr, 1.0, 0.5, lbm.LBM_EOS_PR, 0.344))
        s = orc.Setup(nx=4, ny=4, eos="pr", a=2 / 49, b=2 / 21, T_over_Tc=tr)
        g2, l2, p2 = s.coexistence()
        assert abs(Tc / (s.T / tr) - 1) < 1e-12
        assert abs(g / g2 - 1) < 1e-10 and abs(l / l2 - 1) < 1e-12 and abs(p / p2 - 1) < 1e-10


def test_binding_constants_match_header_enums(lbm):
    """Every enumerator of include/lbm.h that the binding exports has the
    header's value (options, statuses, EOS and collision kinds)."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "lbm.h")).read(), flags=re.S)
    found = 0
    for body in re.findall(r"typedef\s+enum\s*\{(.*?)\}", text, flags=re.S):
        value = -1
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            m = re.match(r"(LBM_[A-Z0-9_]+)\s*(?:=\s*(-?\d+))?$", item)
            assert m, item
            value = int(m.group(2)) if m.group(2) is not None else value + 1
            if hasattr(lbm, m.group(1)):
                assert getattr(lbm, m.group(1)) == value, m.group(1)
                found += 1
    assert found >= 15
    assert (lbm.LBM_OPT_ROWS2, lbm.LBM_OPT_TMA, lbm.LBM_OPT_PREFETCH, lbm.LBM_OPT_GENERAL) == (6, 7, 8, 9)


def test_noalloc_rejects_misaligned_buffers_without_a_launch(lbm):
    # pointers that do not hold whole values of the grid precision are refused
    # during argument checking, before any CUDA call (this runs without a GPU)
    g = lbm.lbm_grid(64, 32, 1, 0, 32)
    g64 = lbm.lbm_grid(64, 32, 1, 0, 64)
    e = lbm.lbm_eos(1.0, 4.0, 1.0, 0.8, 1.0, 0.5)
    good, bad2, bad4 = 0x10000, 0x20002, 0x30004
    assert lbm.lbm_step_noalloc(g, e, 1.0, 0.0, None, bad2, good, 0) == lbm.LBM_ERR_ARG
    assert lbm.lbm_step_noalloc(g, e, 1.0, 0.0, None, good, bad2, 0) == lbm.LBM_ERR_ARG
    assert lbm.lbm_step_noalloc(g64, e, 1.0, 0.0, None, bad4, good, 0) == lbm.LBM_ERR_ARG
    assert lbm.lbm_step_noalloc(g, e, 1.0, 0.0, None, good, 0x40000, 0, diag_ptr=bad4) == lbm.LBM_ERR_ARG
    assert lbm.lbm_step_noalloc(g, e, 1.0, 0.0, None, good, 0x40000, 0, err_ptr=bad2) == lbm.LBM_ERR_ARG


def test_fault_injection_param_before_any_cuda_call(lbm, monkeypatch):
    # LBM_FAULT=param fails lbm_init as if the thermodynamics had no solution;
    # the check comes before the first CUDA call, so it runs without a GPU
    g = lbm.lbm_grid(16, 16, 0, 0, 32)
    e = lbm.lbm_eos(1.0, 4.0, 1.0, 0.8, 1.0, 0.5)
    monkeypatch.setenv("LBM_FAULT", "param")
    with pytest.raises(lbm.LBMError) as ei:
        lbm.lbm_init(g, e, 1.0, 0.0, None, np.full((16, 16), 0.1))
    assert ei.value.status == lbm.LBM_ERR_PARAM

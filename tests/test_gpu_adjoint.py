"""Discrete adjoint (lbm_adjoint_*) against central finite differences of the
FP64 oracle.

The objectives are the time-integrated wall loads J_tau = sum_n sum_x tau_w and
J_p = sum_n sum_x p_w over the states that N steps read. The oracle computes
them with its own step; its central differences are the reference
derivatives. Each small case is first checked to be well posed (differences
at h and h/4 agree), because a pressure column's clamped phase weight makes
J piecewise smooth in the pressure drop wherever a neighbour crosses a phase
end point.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def adjm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_08301_gb300 import build
    build.build()
    import paper_2103_08301_gb300.adjoint as m
    return m


# --- cases: geometry, physics, initial profile, parameters ------------------

def _case(name):
    if name == "periodic_body_force":
        # two-phase airway in a channel periodic in x, driven by a body force
        return dict(nx=96, ny=40, walls=True, bc_x=False, T_over_Tc=0.85, kappa=0.5, steps=200,
                    dp=0.0, gx=2e-6, film=5.0, plug_x=24.0, plug_len=20.0, noise=1e-3, p_ref=None,
                    scale=(1.0, 1.0), params=("gx", "film", "plug_len"))
    if name == "supercritical_columns":
        # single phase above Tc between pressure columns: no phase weight
        return dict(nx=64, ny=24, walls=True, bc_x=True, T_over_Tc=1.1, kappa=0.5, steps=150,
                    dp=2e-4, gx=0.0, film=4.0, plug_x=20.0, plug_len=12.0, noise=1e-3, p_ref="mid",
                    scale=(0.15, 0.12), params=("dp", "film", "plug_len", "gx"))
    if name == "two_phase_columns":
        # film and plug between pressure columns, short horizon, interface rows
        # inside the phase weight's linear range
        return dict(nx=96, ny=40, walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5, steps=40,
                    dp=1e-3, gx=0.0, film=5.0, plug_x=30.0, plug_len=16.0, noise=0.0, p_ref=None,
                    scale=(1.02, 0.9), params=("dp", "film", "plug_len"))
    if name == "mrt_periodic_body_force":
        # the first case with MRT collision (every rate away from 1/tau)
        c = _case("periodic_body_force")
        c.update(tau=1.2, coll=dict(collision="mrt", s_e=1.2, s_eps=1.54, s_q=1.1, s_j=1.0, s_nu=1 / 1.2))
        return c
    raise KeyError(name)


def _setup(orc, c, dp=None, gx=None):
    s0 = orc.Setup(nx=c["nx"], ny=c["ny"], walls=c["walls"], bc_x=False, T_over_Tc=c["T_over_Tc"],
                   kappa=c["kappa"])
    p_ref = None
    if c["p_ref"] == "mid":
        p_ref = orc.cs_p0(s0.a, s0.b, s0.R, s0.T, 0.13)
    s = orc.Setup(nx=c["nx"], ny=c["ny"], walls=c["walls"], bc_x=c["bc_x"], T_over_Tc=c["T_over_Tc"],
                  kappa=c["kappa"], dp=c["dp"] if dp is None else dp, gx=c["gx"] if gx is None else gx,
                  p_ref=p_ref, tau=c.get("tau", 1.0), **c.get("coll", {}))
    return s, p_ref


def _phases(orc, c, s):
    """(liquid, gas) densities of the initial profile: scaled Maxwell values
    below Tc, the case's absolute values above."""
    if c["T_over_Tc"] < 1.0:
        g, l, _ = s.coexistence()
        return l * c["scale"][0], g * c["scale"][1]
    return c["scale"]


def _rho0(orc, c, s, film=None, plug_len=None):
    l, g = _phases(orc, c, s)
    return synth.airway_rho0(c["nx"], c["ny"], c["film"] if film is None else film, c["plug_x"],
                             c["plug_len"] if plug_len is None else plug_len, l, g, noise=c["noise"], seed=1)


def _oracle_J(orc, c, **kw):
    s, _ = _setup(orc, c, dp=kw.get("dp"), gx=kw.get("gx"))
    r0 = _rho0(orc, c, s, film=kw.get("film"), plug_len=kw.get("plug_len"))
    _, d = orc.run(s, orc.init(s, r0), c["steps"])
    return np.array([d["J"], d["Jp"]])


_STEP = {"dp": 1e-6, "gx": 1e-8, "film": 1e-4, "plug_len": 1e-4}


def _oracle_fd(orc, c, p, h):
    x0 = c[p]
    return (_oracle_J(orc, c, **{p: x0 + h}) - _oracle_J(orc, c, **{p: x0 - h})) / (2 * h)


_FD_CACHE = {}


def oracle_fd(orc, name, p):
    """Central differences of (J_tau, J_p) at steps h and h/4, Richardson-
    extrapolated (error O(h^4)); the two must agree to 1e-5, which a kink
    between them would break."""
    key = (name, p)
    if key not in _FD_CACHE:
        c = _case(name)
        h = _STEP[p]
        d1, d2 = _oracle_fd(orc, c, p, h), _oracle_fd(orc, c, p, h / 4)
        scale = np.abs(d2).max()
        assert np.abs(d1 - d2).max() <= 1e-5 * scale, (name, p, d1, d2)
        _FD_CACHE[key] = (16.0 * d2 - d1) / 15.0
    return _FD_CACHE[key]


def _adjoint(adjm, orc, c, block_steps=0):
    s, p_ref = _setup(orc, c)
    adj = adjm.Adjoint(c["nx"], c["ny"], c["steps"], walls=c["walls"], bc_x=c["bc_x"], T_over_Tc=c["T_over_Tc"],
                       kappa=c["kappa"], p_ref=p_ref, block_steps=block_steps, tau=c.get("tau", 1.0),
                       **c.get("coll", {}))
    r0 = _rho0(orc, c, s)
    J = adj.forward(r0, dp=c["dp"], gx=c["gx"])
    return adj, s, J


def _grads(adjm, orc, c, adj, w_tau, w_p):
    import paper_2103_08301_gb300 as lbm
    s, _ = _setup(orc, c)
    g_rho0, gd = adj.backward(w_tau, w_p)
    l, g = _phases(orc, c, s)
    d_film, d_plug = lbm.lbm_airway_rho0_tangent(c["nx"], c["ny"], c["film"], c["plug_x"], c["plug_len"], l, g)
    return {"dp": gd["dp"], "gx": gd["gx"], "film": float((g_rho0 * d_film).sum()),
            "plug_len": float((g_rho0 * d_plug).sum())}, g_rho0


CASES = ["periodic_body_force", "supercritical_columns", "two_phase_columns", "mrt_periodic_body_force"]


@pytest.mark.parametrize("name", CASES)
def test_objective_matches_oracle(adjm, orc, name):
    c = _case(name)
    adj, s, J = _adjoint(adjm, orc, c)
    ref = _oracle_J(orc, c)
    with adj:
        assert abs(J[0] - ref[0]) <= 1e-10 * np.abs(ref[0]) + 1e-13
        assert abs(J[1] - ref[1]) <= 1e-11 * np.abs(ref[1])


@pytest.mark.parametrize("name", CASES)
def test_gradients_match_oracle_finite_differences(adjm, orc, name):
    c = _case(name)
    adj, _, _ = _adjoint(adjm, orc, c)
    with adj:
        per_w = [_grads(adjm, orc, c, adj, 1.0, 0.0)[0], _grads(adjm, orc, c, adj, 0.0, 1.0)[0]]
    for p in c["params"]:
        fd = oracle_fd(orc, name, p)
        for k in range(2):
            got = per_w[k][p]
            assert abs(got - fd[k]) <= 1e-6 * abs(fd[k]) + 1e-9 * np.abs(fd).max(), (name, p, k, got, fd[k])


def test_gradient_independent_of_checkpoint_blocks(adjm, orc):
    c = _case("two_phase_columns")
    out = []
    for K in (1, 7, 0, c["steps"]):
        adj, _, J = _adjoint(adjm, orc, c, block_steps=K)
        with adj:
            g, gd = adj.backward(0.7, -0.3)
        out.append((J, g, gd))
    for J, g, gd in out[1:]:
        assert J == out[0][0]
        assert np.array_equal(g, out[0][1]) and gd == out[0][2]


def test_backward_is_linear_in_the_seeds(adjm, orc):
    c = _case("periodic_body_force")
    adj, _, _ = _adjoint(adjm, orc, c)
    with adj:
        g1, d1 = adj.backward(1.0, 0.0)
        g2, d2 = adj.backward(0.0, 1.0)
        g3, d3 = adj.backward(2.0, -3.0)
    assert np.abs(g3 - (2 * g1 - 3 * g2)).max() <= 1e-12 * np.abs(g3).max()
    assert d3["gx"] == pytest.approx(2 * d1["gx"] - 3 * d2["gx"], rel=1e-12)


def test_autograd_chain_film_plug_and_pressure_drop(adjm, orc):
    import torch
    c = _case("two_phase_columns")
    s, p_ref = _setup(orc, c)
    l, g = _phases(orc, c, s)
    dev = "cuda"
    film = torch.tensor(c["film"], dtype=torch.float64, requires_grad=True)
    plug = torch.tensor(c["plug_len"], dtype=torch.float64, requires_grad=True)
    dp = torch.tensor(c["dp"], dtype=torch.float64, requires_grad=True)
    with adjm.Adjoint(c["nx"], c["ny"], c["steps"], walls=True, bc_x=True, T_over_Tc=c["T_over_Tc"],
                      kappa=c["kappa"]) as adj:
        rho0 = adjm.AirwayProfile.apply(film, plug, c["nx"], c["ny"], c["plug_x"], l, g, 4.0, c["noise"], 1, dev)
        J_tau, J_p = adjm.WallLoads.apply(adj, rho0, dp)
        (J_tau + 0.5 * J_p).backward()
    for p, t in (("dp", dp), ("film", film), ("plug_len", plug)):
        fd = oracle_fd(orc, "two_phase_columns", p)
        ref = fd[0] + 0.5 * fd[1]
        assert abs(t.grad.item() - ref) <= 1e-6 * abs(ref) + 1e-9 * np.abs(fd).max(), (p, t.grad.item(), ref)


_AIRWAY_J = {}


@pytest.mark.parametrize("precision,reverse", [(64, 64), (32, 64), (32, 32)])
def test_airway_workload_gradients_2000_steps(adjm, orc, precision, reverse):
    # the airway workload: 512 x 128 channel, film 6, plug 48 at x = 128,
    # 0.85 Tc, dp = 1e-3, noise 1e-3, 2000 FP64 steps. J is smooth in film
    # thickness and plug length; central differences of the oracle (step 1e-3)
    # are the reference. In dp the column phase weight's clamp leaves kinks
    # (differences move by ~1e-3 between steps 1e-6 and 1e-7), so the dp
    # reference is the difference at step 1e-7 and the bound is the 1e-3 the
    # method targets. precision = 32: FP32 forward and checkpoints (every 100
    # steps), FP64 reverse; J within 1e-5 of the FP64 oracle's, gradients within
    # the same 1e-3 of its central differences. reverse = 32: the reverse sweep
    # and the objective's per-step terms in FP32 as well (sums over steps in
    # FP64), held to the same bounds.
    nx, ny, steps = 512, 128, 2000
    kw = dict(walls=True, bc_x=True, T_over_Tc=0.85, kappa=0.5)
    g, l, _ = orc.Setup(nx=nx, ny=ny, dp=1e-3, **kw).coexistence()

    def J(film=6.0, plug=48.0, dp=1e-3):  # the oracle's (J_tau, J_p), cached over both precisions
        key = (film, plug, dp)
        if key not in _AIRWAY_J:
            s = orc.Setup(nx=nx, ny=ny, dp=dp, **kw)
            r0 = synth.airway_rho0(nx, ny, film, 128, plug, l, g, noise=1e-3, seed=1)
            _, d = orc.run(s, orc.init(s, r0), steps)
            _AIRWAY_J[key] = np.array([d["J"], d["Jp"]])
        return _AIRWAY_J[key]

    import paper_2103_08301_gb300 as lbm
    block = 100 if precision == 32 else 0
    with adjm.Adjoint(nx, ny, steps, precision=precision, reverse_precision=reverse, block_steps=block,
                      **kw) as adj:
        r0 = synth.airway_rho0(nx, ny, 6.0, 128, 48.0, l, g, noise=1e-3, seed=1)
        Jg = adj.forward(r0, dp=1e-3)
        grads = [adj.backward(1.0, 0.0), adj.backward(0.0, 1.0)]
    ref = J()
    tol = (1e-9, 1e-11) if precision == 64 else (1e-5, 1e-5)
    assert abs(Jg[0] / ref[0] - 1) < tol[0] and abs(Jg[1] / ref[1] - 1) < tol[1], (Jg, ref)
    d_film, d_plug = lbm.lbm_airway_rho0_tangent(nx, ny, 6.0, 128, 48.0, l, g)
    h = 1e-3
    fd_film = (J(film=6.0 + h) - J(film=6.0 - h)) / (2 * h)
    fd_plug = (J(plug=48.0 + h) - J(plug=48.0 - h)) / (2 * h)
    fd_dp = (J(dp=1e-3 + 1e-7) - J(dp=1e-3 - 1e-7)) / 2e-7
    for k in range(2):
        gr = grads[k][0]
        got_f, got_p = float((gr * d_film).sum()), float((gr * d_plug).sum())
        assert abs(got_f - fd_film[k]) <= 1e-3 * abs(fd_film[k]), ("film", k, got_f, fd_film[k])
        assert abs(got_p - fd_plug[k]) <= 1e-3 * abs(fd_plug[k]), ("plug", k, got_p, fd_plug[k])
        got_dp = grads[k][1]["dp"]
        assert abs(got_dp - fd_dp[k]) <= 1e-3 * abs(fd_dp[k]), ("dp", k, got_dp, fd_dp[k])


def _node_fd(orc, c, s, r0, x, y, h):
    """Central difference of the oracle's (J_tau, J_p) in the initial density of node (x, y)."""
    def J(r):
        _, d = orc.run(s, orc.init(s, r), c["steps"])
        return np.array([d["J"], d["Jp"]])
    rp, rm = r0.copy(), r0.copy()
    rp[y, x] += h
    rm[y, x] -= h
    return (J(rp) - J(rm)) / (2 * h)


@pytest.mark.parametrize("name", ["two_phase_columns", "periodic_body_force"])
def test_per_node_density_gradient_matches_oracle(adjm, orc, name):
    """dJ/drho0 at single nodes against Richardson-extrapolated central
    differences of the oracle (steps 1e-5 and 2.5e-6, which agree to 1e-5, so
    no kink lies between them): interior bulk and interface nodes, the first
    fluid rows next to both walls, a wall-film node, the nodes next to the
    inlet and outlet columns and the column nodes themselves (zero where
    pressure columns overwrite them, nonzero in the periodic channel). Solid
    wall-row nodes are ignored by the step, so both gradients are zero there."""
    c = _case(name)
    nx, ny = c["nx"], c["ny"]
    adj, s, _ = _adjoint(adjm, orc, c)
    with adj:
        grads = [adj.backward(1.0, 0.0)[0], adj.backward(0.0, 1.0)[0]]
    r0 = _rho0(orc, c, s)
    interior = [(48, 20), (30, 20), (70, 3)]
    wall_adjacent = [(48, 1), (40, ny - 2), (nx - 3, 1)]
    column = [(1, 20), (nx - 2, 10), (0, 20), (nx - 1, 5)]
    fd = {}
    for (x, y) in interior + wall_adjacent + column:
        d1 = _node_fd(orc, c, s, r0, x, y, 1e-5)
        d2 = _node_fd(orc, c, s, r0, x, y, 2.5e-6)
        assert np.abs(d1 - d2).max() <= 1e-5 * np.abs(d2).max() + 1e-300, ((x, y), d1, d2)
        fd[(x, y)] = (16.0 * d2 - d1) / 15.0
    scale = max(np.abs(v).max() for v in fd.values())
    for (x, y), ref in fd.items():
        for k in range(2):
            got = grads[k][y, x]
            assert abs(got - ref[k]) <= 1e-6 * abs(ref[k]) + 1e-9 * scale, (name, (x, y), k, got, ref[k])
    if c["bc_x"]:
        for k in range(2):
            assert fd[(0, 20)][k] == 0.0 and fd[(nx - 1, 5)][k] == 0.0
            assert np.abs(grads[k][:, 0]).max() <= 1e-12 * scale and np.abs(grads[k][:, -1]).max() <= 1e-12 * scale
    for k in range(2):
        assert np.abs(grads[k][0]).max() <= 1e-12 * scale and np.abs(grads[k][-1]).max() <= 1e-12 * scale


def test_fp32_reverse_sweep_tracks_the_fp64_one(adjm, orc):
    """The FP32 reverse sweep on an FP32 forward against the FP64 sweep on the
    same stored states: per-node dJ/drho0 within 1e-4 of the largest entry and
    the drive gradients within 1e-4 relative (FP32 rounding over 200 reverse
    steps of a two-phase channel under a body force)."""
    c = _case("periodic_body_force")
    s, _ = _setup(orc, c)
    r0 = _rho0(orc, c, s)
    out = {}
    for rev in (64, 32):
        with adjm.Adjoint(c["nx"], c["ny"], c["steps"], walls=True, bc_x=False, T_over_Tc=c["T_over_Tc"],
                          kappa=c["kappa"], precision=32, reverse_precision=rev) as adj:
            J = adj.forward(r0, gx=c["gx"])
            out[rev] = (J, adj.backward(1.0, 0.5))
    (J64, (g64, d64)), (J32, (g32, d32)) = out[64], out[32]
    assert abs(J32[0] / J64[0] - 1) < 1e-5 and abs(J32[1] / J64[1] - 1) < 1e-5
    assert np.abs(g32 - g64).max() <= 1e-4 * np.abs(g64).max()
    assert abs(d32["gx"] / d64["gx"] - 1) < 1e-4

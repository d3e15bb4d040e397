"""Physics pins of the oracle's full time step.

Each test checks the stepping against something the oracle does not compute
itself: an analytic flow, a conservation law, an exact discrete balance
derived by hand from the scheme, the Maxwell construction (solved by scipy),
the continuum surface tension of the free energy (Eq. 2.3) integrated by
scipy, or a symmetry of the wall rule.
"""
import numpy as np
import pytest

import synth

scipy_int = pytest.importorskip("scipy.integrate")

NU1 = 1.0 / 6.0  # kinematic viscosity (tau - 1/2)/3 at tau = 1


def test_uniform_states_are_invariant(orc):
    # rest state, and a uniformly moving state on a periodic box
    for ux, uy in [(0.0, 0.0), (0.03, -0.02)]:
        s = orc.Setup(nx=12, ny=10, T_over_Tc=0.8, kappa=0.5)
        f = np.empty((9, 10, 12))
        f[:] = orc.feq(0.17, ux, uy)[:, None, None]
        g, _ = orc.run(s, f, 50)
        assert np.abs(g - f).max() < 1e-15


@pytest.mark.parametrize("walls", [False, True])
def test_mass_conserved_to_1e12(orc, walls):
    n = 128 if not walls else 96
    s = orc.Setup(nx=n, ny=n, walls=walls, T_over_Tc=0.8, kappa=0.5)
    g, l, _ = s.coexistence()
    rho0 = synth.disk_rho0(n, n, 30, l, g, noise=1e-3, seed=1)
    f = orc.init(s, rho0)
    _, d0 = orc.step(s, f)
    f, d = orc.run(s, f, 10000 if not walls else 4000)
    f, d1 = orc.step(s, f)
    assert abs(d1["mass"] - d0["mass"]) <= 1e-12 * d0["mass"]


def _poiseuille(orc, H):
    rho0 = 0.2
    G = 0.01 * 8 * rho0 * NU1 / H**2
    # supercritical single phase; kappa = 0 and uniform density give F = G
    s = orc.Setup(nx=1, ny=H + 2, walls=True, T_over_Tc=1.5, kappa=0.0, gx=G)
    f = orc.init(s, np.full((H + 2, 1), rho0))
    f, _ = orc.run(s, f, int(14 * H * H / (NU1 * np.pi**2)) + 100)
    fl = orc.fields(s, f)
    y = np.arange(1, H + 1)
    exact = G / (2 * rho0 * NU1) * (y - 0.5) * (H + 0.5 - y)  # no-slip on half-way planes
    v = fl["vx"][1:H + 1, 0]
    return np.abs(v - exact).max() / exact.max(), fl["tau_wall"][:, 0], G * H / 2


def test_poiseuille_profile_and_wall_shear(orc):
    errs, tws = [], []
    for H in (16, 32, 64):
        e, tw, tw_exact = _poiseuille(orc, H)
        errs.append(e)
        tws.append(abs(tw[0] / tw_exact - 1))
        assert abs(tw[0] - tw[1]) < 1e-12 * abs(tw[0])  # both walls, same sign for +x flow
    assert errs[-1] < 1e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5  # second order
    assert tws[-1] < 0.01 and tws[0] > tws[1] > tws[2]          # tau_w -> G H / 2


def _relaxed_slab(orc, T_over_Tc, n=256, steps=40000, kappa=0.5):
    s = orc.Setup(nx=2, ny=n, T_over_Tc=T_over_Tc, kappa=kappa)
    g, l, _ = s.coexistence()
    f = orc.init(s, synth.slab_rho0(2, n, n // 4, 3 * n // 4, l, g, width=4))
    f, _ = orc.run(s, f, steps)
    return s, f, g, l


def test_flat_interface_discrete_balance_at_tau_one(orc):
    """At tau = 1 the post-streaming populations are the equilibria of the upstream
    nodes. For a steady flat interface (v = 0, so u_eq = F / (2 rho)) summing the
    D2Q9 equilibria by e_y gives, exactly, with P = rho/6 + F^2/(8 rho):
        P(y+1) - P(y-1) = F(y)/2 + (F(y-1) + F(y+1))/4.
    A wrong sign or factor in the velocity shift, the collision or the streaming
    breaks this identity."""
    s, f, g, l = _relaxed_slab(orc, 0.8, n=128, steps=60000)
    fl = orc.fields(s, f)
    _, Fy = orc.force(s, f)
    r, F = fl["rho"][:, 0], Fy[:, 0]
    assert np.abs(fl["vy"]).max() < 1e-12
    P = r / 6 + F**2 / (8 * r)
    lhs = np.roll(P, -1) - np.roll(P, 1)
    rhs = F / 2 + (np.roll(F, 1) + np.roll(F, -1)) / 4
    assert np.abs(lhs - rhs).max() < 1e-14
    assert np.abs(F).max() > 1e-2  # the identity is not trivially satisfied


def test_coexistence_converges_to_maxwell_as_interface_widens(orc):
    """Maxwell equal-area densities (scipy-pinned in test_oracle_eos) are reached as
    the interface widens relative to the lattice (T -> Tc); the deviation at
    lower T is a lattice-scale effect of the forcing scheme: the lattice's own
    ideal pressure is a smoothed rho/3 that the central-difference gradient of
    rho/3 does not cancel, and the velocity shift adds F^2/(4 rho) to the
    momentum flux (the exact balance pinned above)."""
    errs = []
    for t in (0.95, 0.98):
        s, f, g, l = _relaxed_slab(orc, t, steps=60000)
        r = orc.fields(s, f)["rho"][:, 0]
        rl, rg = r[128], r[0]
        errs.append(max(abs(rl / l - 1), abs(rg / g - 1)))
    assert errs[1] < 0.015
    assert errs[0] > errs[1]


def test_relaxed_flat_interface_has_equal_bulk_pressures(orc):
    """Momentum balance of a steady flat interface: summing the exact tau = 1
    balance above over y telescopes to (rho_l - rho_g)/3 = sum_y F_y, and with
    F = -grad(k^2 p0 - rho/3) + kappa rho grad(lap rho) the pressure part
    telescopes to -(k^2 p0(rho_l) - rho_l/3) + (k^2 p0(rho_g) - rho_g/3) while
    sum_y rho_y (L_{y+1} - L_{y-1}) / 2 vanishes identically for a profile in
    y alone (by parts it is minus the sum of (a_{y+1}^2 - a_y^2)/2 with a_y =
    rho_y - rho_{y-1}). Hence the two bulk phases carry the same EOS pressure,
    p0(rho_g*) = p0(rho_l*), although neither density is Maxwell's: this
    common pressure is the method's own saturation pressure."""
    s, f, g, l = _relaxed_slab(orc, 0.85, n=192, steps=40000)
    r = orc.fields(s, f)["rho"][:, 0]
    rg, rl = r[0], r[96]
    pg = orc.cs_p0(s.a, s.b, s.R, s.T, rg)
    pl = orc.cs_p0(s.a, s.b, s.R, s.T, rl)
    assert abs(pl / pg - 1) < 1e-6
    _, _, psat = s.coexistence()
    # at this interface width (about 5 nodes) both lie well below Maxwell's
    assert pg < 0.8 * psat and rg < 0.75 * g


@pytest.mark.parametrize("t", [0.85, 0.9])
def test_flat_interface_matches_maxwell_at_the_cancelling_relaxation_time(orc, t):
    """The two lattice terms that move the method's coexistence off Maxwell's
    (the smoothed lattice ideal pressure against the central-difference
    gradient of rho/3, and the velocity shift's F^2/(4 rho) flux, whose weight
    follows tau) cancel near tau = 1.36: there the flat interface's bulk
    densities are Maxwell's equal-area densities (solved by scipy in
    test_oracle_eos) within 1%, at 0.85 and 0.9 Tc; at tau = 1 the vapour is
    13-31% too thin at these temperatures."""
    for tau, within in ((1.36, 0.01), (1.0, None)):
        s = orc.Setup(nx=2, ny=192, T_over_Tc=t, kappa=0.5, tau=tau)
        g, l, _ = s.coexistence()
        f = orc.init(s, synth.slab_rho0(2, 192, 48, 144, l, g, width=4))
        f, _ = orc.run(s, f, 60000)
        r = orc.fields(s, f)["rho"][:, 0]
        eg, el = r[0] / g - 1, r[96] / l - 1
        if within:
            assert abs(eg) < within and abs(el) < within, (t, tau, eg, el)
        else:
            assert eg < -0.1, (t, tau, eg)


def _sigma_theory(orc, s):
    """sigma = k sqrt(2 kappa) int_{rho_g}^{rho_l} sqrt(dOmega) drho with
    dOmega(rho) = int_{rho_g}^{rho} (mu(r) - mu_sat) dr and mu(r) - mu_sat =
    int_{rho_g}^{r} p0'(t)/t dt: the flat-interface tension of the square-gradient
    free energy of Eq. 2.3 scaled to the mesh by Eq. 2.14."""
    g, l, _ = s.coexistence()
    T = s.T

    def dmu(r):
        return scipy_int.quad(lambda t: orc.cs_dp0(s.a, s.b, s.R, T, t) / t, g, r,
                              epsabs=1e-15, epsrel=1e-12)[0]

    rs = np.linspace(g, l, 801)
    dm = np.array([dmu(r) for r in rs])
    dOm = np.concatenate([[0.0], np.cumsum(0.5 * (dm[1:] + dm[:-1]) * np.diff(rs))])
    integ = np.sqrt(np.maximum(dOm, 0.0))
    return s.k * np.sqrt(2 * s.kappa) * np.trapezoid(integ, rs)


def test_laplace_law(orc):
    n, pts = 96, []
    s = None
    for R0 in (14, 18, 22, 26, 30):
        s = orc.Setup(nx=n, ny=n, T_over_Tc=0.8, kappa=0.5)
        g, l, _ = s.coexistence()
        f = orc.init(s, synth.disk_rho0(n, n, R0, l, g))
        f, _ = orc.run(s, f, 6000)
        r = orc.fields(s, f)["rho"]
        rin, rout = r[n // 2, n // 2], r[0, 0]
        dp = s.k**2 * (orc.cs_p0(s.a, s.b, s.R, s.T, rin) - orc.cs_p0(s.a, s.b, s.R, s.T, rout))
        Req = np.sqrt(((r - rout) / (rin - rout)).sum() / np.pi)  # equimolar radius
        pts.append((1 / Req, dp))
    x, y = np.array(pts).T
    m, c = np.polyfit(x, y, 1)
    r2 = 1 - ((y - (m * x + c)) ** 2).sum() / ((y - y.mean()) ** 2).sum()
    assert r2 > 0.999
    assert abs(c) < 0.03 * y.min()
    assert abs(m / _sigma_theory(orc, s) - 1) < 0.03


def test_neutral_wetting_gives_ninety_degrees(orc):
    nx, ny = 128, 64
    s = orc.Setup(nx=nx, ny=ny, walls=True, T_over_Tc=0.8, kappa=0.5)
    g, l, _ = s.coexistence()
    f = orc.init(s, synth.disk_rho0(nx, ny, 22, l, g, centre=(nx / 2, 0.5)))
    f, _ = orc.run(s, f, 8000)
    r = orc.fields(s, f)["rho"]
    mid = 0.5 * (r[1, nx // 2] + r[ny - 2, 0])
    col = r[1:ny - 1, nx // 2]
    i = int(np.argmax(col < mid))
    h = (i + (col[i - 1] - mid) / (col[i - 1] - col[i])) - 0.5 + 0.0  # from the wall plane
    row = r[1, :]
    ins = np.where(row > mid)[0]
    xl = ins[0] - (row[ins[0]] - mid) / (row[ins[0]] - row[ins[0] - 1])
    xr = ins[-1] + (row[ins[-1]] - mid) / (row[ins[-1]] - row[ins[-1] + 1])
    theta = 2 * np.degrees(np.arctan(h / (0.5 * (xr - xl))))  # circular cap: tan(theta/2) = h/a
    assert abs(theta - 90.0) < 3.0


def test_pressure_columns_drive_poiseuille_flow(orc):
    nx, ny, H, dp = 256, 34, 32, 2e-5
    Tc, _ = orc.cs_critical()
    pref = orc.cs_p0(1.0, 4.0, 1.0, 1.5 * Tc, 0.2)
    s = orc.Setup(nx=nx, ny=ny, walls=True, bc_x=True, T_over_Tc=1.5, kappa=0.0, dp=dp, p_ref=pref)
    # imposed densities sit on the EOS at p_ref +- dp/2
    assert abs(orc.cs_p0(s.a, s.b, s.R, s.T, s.rho_in) - (pref + dp / 2)) < 1e-15
    assert abs(orc.cs_p0(s.a, s.b, s.R, s.T, s.rho_out) - (pref - dp / 2)) < 1e-15
    f = orc.init(s, np.full((ny, nx), 0.2))
    f, _ = orc.run(s, f, 20000)
    fl = orc.fields(s, f)
    y = np.arange(1, ny - 1)
    v = fl["vx"][1:ny - 1, nx // 2]
    shape = (y - 0.5) * (H + 0.5 - y)
    c = (v * shape).sum() / (shape * shape).sum()
    assert np.abs(v - c * shape).max() < 2e-3 * v.max()
    G = dp / (nx - 1)  # pressure gradient between the column centres
    assert abs(c / (G / (2 * fl["rho"][ny // 2, nx // 2] * NU1)) - 1) < 0.01


def test_wall_pressure_sum_of_resting_channel(orc):
    # A uniform channel at rest between walls (periodic in x) is invariant;
    # with no density gradient Eq. 2.4 leaves p_w = k^2 p0(rho) at every wall
    # column, so J_p = steps * 2 * nx * k^2 p0(rho) and the wall shear vanishes.
    for k in (1.0, 0.7):
        s = orc.Setup(nx=10, ny=9, walls=True, T_over_Tc=0.9, kappa=0.5, k=k)
        rho = 0.12
        f = orc.init(s, np.full((9, 10), rho))
        _, d = orc.run(s, f, 7)
        p0 = orc.cs_p0(s.a, s.b, s.R, s.T, rho)
        assert d["Jp"] == pytest.approx(7 * 2 * 10 * k * k * p0, rel=1e-13)
        assert abs(d["J"]) < 1e-15


def test_body_force_drive_with_extrapolated_ends(orc):
    # The paper's drive (Sec. 2.2): a body force G along the channel, the ends
    # held at one pressure (dp = 0) by non-equilibrium extrapolation. Single
    # phase, kappa = 0: the developed flow is Poiseuille on the half-way wall
    # planes with amplitude (G - dp/dx) / (2 rho nu), dp/dx the small pressure
    # gradient (p = k^2 p0(rho)) the extrapolated ends leave in the bulk.
    nx, ny, H, G = 128, 34, 32, 2e-7
    Tc, _ = orc.cs_critical()
    pref = orc.cs_p0(1.0, 4.0, 1.0, 1.5 * Tc, 0.2)
    s = orc.Setup(nx=nx, ny=ny, walls=True, bc_x=True, T_over_Tc=1.5, kappa=0.0, dp=0.0, p_ref=pref, gx=G)
    assert s.rho_in == s.rho_out
    f = orc.init(s, np.full((ny, nx), s.rho_in))
    f, _ = orc.run(s, f, 20000)
    fl = orc.fields(s, f)
    y = np.arange(1, ny - 1)
    shape = (y - 0.5) * (H + 0.5 - y)
    p1, p3 = (orc.cs_p0(s.a, s.b, s.R, s.T, float(fl["rho"][ny // 2, x])) for x in (nx // 4, 3 * nx // 4))
    dpdx = (p3 - p1) / (nx // 2)
    assert 0 < dpdx < 0.02 * G  # a slight adverse gradient
    for x in (nx // 4, nx // 2, 3 * nx // 4):
        v = fl["vx"][1:ny - 1, x]
        exact = (G - dpdx) / (2 * fl["rho"][ny // 2, x] * NU1) * shape
        assert np.abs(v - exact).max() < 1e-3 * exact.max()

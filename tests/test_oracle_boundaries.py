"""Pins of the oracle's boundary arithmetic against independent routes.

Covered here, each by a check that a sign, branch, index or depth error fails:
  - the EOS branch roots a pressure column takes (liquid root, gas root, and
    the spinodal density a pressure beyond a branch's end saturates to),
    against brentq on sympy's Carnahan-Starling / Peng-Robinson p0 (Eq. 2.18);
  - the column density of the step (R6: the EOS root at p_ref +- dp/2 on the
    branch of the interior neighbour's phase, blended linearly between the
    Maxwell densities and clamped), read back through the oracle's fields;
  - one step of the non-equilibrium extrapolation of the columns on a hand-
    built two-phase state, in closed form (f* = f_eq(rho_b, v_f) +
    (1 - 1/tau)(f(x_f) - f_eq(rho_f, v_f)), then streamed into the lattice);
  - the kappa terms of the wall pressure (Eq. 2.4, p_w = k^2 p0 - kappa rho
    lap rho - kappa/2 |grad rho|^2) on long-wave profiles, against analytic
    derivatives with second-order convergence;
  - the wetting offset of the mirrored ghost densities (R7): closed-form
    forces next to a wall of a uniform liquid, and the sessile-drop contact
    angle moving away from 90 degrees in opposite directions for the two
    signs of the offset.
"""
import numpy as np
import pytest

import synth

sympy = pytest.importorskip("sympy")
scipy_opt = pytest.importorskip("scipy.optimize")
scipy_int = pytest.importorskip("scipy.integrate")

# D2Q9 as the paper's nine-entry MRT matrix implies (Sec. 2.1)
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def _eos_functions(s):
    """p0 and dp0/drho of the set-up's EOS from sympy (independent of the oracle's C)."""
    rho = sympy.symbols("rho", positive=True)
    if s.eos == "cs":
        eta = sympy.Float(s.b, 30) * rho / 4
        p = rho * s.R * sympy.Float(s.T, 30) * (1 + eta + eta**2 - eta**3) / (1 - eta) ** 3 - s.a * rho**2
        rmax = 4.0 / s.b
    else:
        b = sympy.Float(s.b, 30)
        p = rho * s.R * sympy.Float(s.T, 30) / (1 - b * rho) - sympy.Float(s.aalpha, 30) * rho**2 / (
            1 + 2 * b * rho - b**2 * rho**2)
        rmax = 1.0 / s.b
    return sympy.lambdify(rho, p), sympy.lambdify(rho, sympy.diff(p, rho)), rmax


def _branches(s):
    """(p0, dp0, s1, s2, rmax): the spinodals s1 < s2 by brentq on sympy's dp0/drho."""
    pf, dpf, rmax = _eos_functions(s)
    # a bracket split point between the spinodals: the maximum of dp0 lies there
    grid = np.linspace(rmax * 1e-4, rmax * 0.999, 4001)
    d = np.array([dpf(r) for r in grid])
    assert (d < 0).any(), "no spinodal region"
    neg = np.where(d < 0)[0]
    s1 = scipy_opt.brentq(dpf, grid[neg[0] - 1], grid[neg[0]], xtol=1e-16)
    s2 = scipy_opt.brentq(dpf, grid[neg[-1]], grid[neg[-1] + 1], xtol=1e-16)
    return pf, dpf, s1, s2, rmax


def _maxwell(pf, s1, s2, rmax):
    """Equal area in specific volume: int p dv over [v_l, v_g] = p_sat (v_g - v_l)."""
    def roots(ps):
        return (scipy_opt.brentq(lambda r: pf(r) - ps, 1e-14, s1, xtol=1e-17),
                scipy_opt.brentq(lambda r: pf(r) - ps, s2, rmax * (1 - 1e-12), xtol=1e-17))

    def area(ps):
        rg, rl = roots(ps)
        val, _ = scipy_int.quad(lambda v: pf(1.0 / v), 1.0 / rl, 1.0 / rg, epsabs=1e-16, epsrel=1e-13, limit=300)
        return val - ps * (1.0 / rg - 1.0 / rl)

    lo = max(pf(s2), 1e-14) * (1 + 1e-10)
    ps = scipy_opt.brentq(area, lo, pf(s1) * (1 - 1e-10), xtol=1e-18, rtol=1e-14)
    rg, rl = roots(ps)
    return rg, rl, ps


def _branch_root(pf, p, lo, hi):
    return scipy_opt.brentq(lambda r: pf(r) - p, lo, hi, xtol=1e-17)


CS = dict(eos="cs")
PR = dict(eos="pr", a=2 / 49, b=2 / 21, omega=0.344)


@pytest.mark.parametrize("kw,t", [(CS, 0.6), (CS, 0.85), (CS, 0.95), (PR, 0.6), (PR, 0.8)])
def test_liquid_root_and_saturation_branches(orc, kw, t):
    s = orc.Setup(nx=4, ny=4, T_over_Tc=t, kappa=0.5, **kw)
    e = s.eos_spec()
    pf, dpf, s1, s2, rmax = _branches(s)
    g, l, ps = _maxwell(pf, s1, s2, rmax)
    pl_end, pg_end = pf(s2), pf(s1)  # the liquid branch ends below at pl_end, the gas branch above at pg_end
    # liquid branch: inversion with p0' > 0 and rho above the liquid spinodal
    # (between the branch ends three densities share a pressure: the middle one
    # lies on the unstable branch, s1 < rho < s2, and must never be returned)
    targets = [ps, 0.5 * (max(pl_end, 0.0) + ps), 1.5 * ps, 3.0 * ps, ps + 0.2 * (pg_end - ps),
               pl_end + 0.02 * (pg_end - pl_end), pl_end + 0.3 * (pg_end - pl_end)]
    for p in targets:
        r = orc.eos_liquid_root(e, p)
        ref = _branch_root(pf, p, s2, rmax * (1 - 1e-12))
        assert abs(r - ref) <= 1e-11 * ref, (p, r, ref)
        assert r > s2 and dpf(r) > 0
        rc, sat = orc.eos_column_density(e, True, p)
        assert not sat and abs(rc - ref) <= 1e-11 * ref
        if s.eos == "cs":
            assert abs(orc.liquid_root(s.a, s.b, s.R, s.T, p) - ref) <= 1e-11 * ref
    assert abs(orc.eos_liquid_root(e, ps) - l) <= 1e-8 * l  # Maxwell liquid at p_sat
    # gas branch below its end
    for p in (0.3 * ps, ps, 0.5 * (ps + pg_end)):
        r = orc.eos_gas_root(e, p)
        ref = _branch_root(pf, p, 1e-14, s1)
        assert abs(r - ref) <= 1e-11 * ref and r < s1 and dpf(r) > 0
    # beyond a branch's end the column saturates at that branch's spinodal
    rg_sat, sat = orc.eos_column_density(e, False, pg_end * 1.05)
    assert sat and abs(rg_sat - s1) <= 1e-9 * s1
    rg_in, sat = orc.eos_column_density(e, False, pg_end * 0.95)
    assert not sat and rg_in < s1
    if pl_end > 0:
        rl_sat, sat = orc.eos_column_density(e, True, pl_end * 0.9)
        assert sat and abs(rl_sat - s2) <= 1e-9 * s2
    with pytest.raises(ValueError):
        orc.eos_liquid_root(e, pl_end - abs(pl_end) * 0.01 - 1e-9)
    with pytest.raises(ValueError):
        orc.eos_column_density(e, False, -1e-4)  # no gas density at a non-positive pressure


def _column_case(orc, T, k, dp, ny=9):
    """A periodic-y strip with pressure columns whose interior neighbours carry a
    chosen density per row; returns the set-up, the state and those densities."""
    nx = 6
    s = orc.Setup(nx=nx, ny=ny, bc_x=True, T_over_Tc=T, k=k, kappa=0.5, dp=dp)
    pf, dpf, s1, s2, rmax = _branches(s)
    g, l, ps = _maxwell(pf, s1, s2, rmax)
    fr = np.array([-0.03, 0.0, 0.1, 0.25, 0.5, 0.8, 1.0, 1.04, 0.6])[:ny]
    rho = np.full((ny, nx), 0.5 * (g + l))
    rho[:, 1] = g + fr * (l - g)
    rho[:, nx - 2] = g + fr[::-1] * (l - g)
    f = orc.init(s, rho)
    return s, f, rho, (pf, s1, s2, rmax, g, l, ps)


@pytest.mark.parametrize("T,k,dp", [(0.85, 1.0, 4e-4), (0.85, 0.9, 6e-4), (0.95, 1.0, 1.4e-3)])
def test_column_density_blend_in_the_step(orc, T, k, dp):
    s, f, rho, (pf, s1, s2, rmax, g, l, ps) = _column_case(orc, T, k, dp)
    got = orc.fields(s, f)["rho"]
    p_ref = k * k * ps  # the default reference: the mesh pressure k^2 p_sat
    for side, xf, xb, sign in ((0, 1, 0, +1), (1, s.nx - 2, s.nx - 1, -1)):
        p = (p_ref + sign * 0.5 * dp) / (k * k)  # EOS pressure of the inlet (+) / outlet (-) column
        gas = s1 if p >= pf(s1) else _branch_root(pf, p, 1e-14, s1)
        liq = s2 if p <= pf(s2) else _branch_root(pf, p, s2, rmax * (1 - 1e-12))
        theta = np.clip((rho[:, xf] - g) / (l - g), 0.0, 1.0)
        want = gas + theta * (liq - gas)
        assert np.abs(got[:, xb] - want).max() <= 1e-10 * want.max(), (side, got[:, xb], want)
        # the end points of the blend are the branch roots themselves
        assert abs(got[1, xb] - gas) <= 1e-10 * gas if side == 0 else True
    if T == 0.95:
        # inlet gas and outlet liquid both past their branch ends: spinodal densities
        assert abs(got[1, 0] - s1) <= 1e-9 * s1
        assert abs(got[2, s.nx - 1] - s2) <= 1e-9 * s2  # row 2 of the outlet has theta = 1


def _feq(rho, ux, uy):
    eu = EX * ux + EY * uy
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    return rho * w * (1 + 3 * eu + 4.5 * eu**2 - 1.5 * (ux * ux + uy * uy))


@pytest.mark.parametrize("tau", [1.0, 1.35])
def test_column_extrapolation_one_step_closed_form(orc, tau):
    """Two-phase neighbours, a moving state with a non-equilibrium part: after one
    step the populations the columns push into the lattice are
    f*_i(x_b) = f_eq_i(rho_b, v_f) + (1 - 1/tau)(f_i(x_f) - f_eq_i(rho_f, v_f)),
    v_f = u_f + F_f / (2 rho_f) (Sec. 2.1 velocity), and the inflow slots of the
    columns themselves are left as they were."""
    nx, ny = 7, 4
    s = orc.Setup(nx=nx, ny=ny, bc_x=True, T_over_Tc=0.85, kappa=0.5, tau=tau, dp=5e-4)
    g, l, _ = s.coexistence()
    rho_x = np.array([0.1, g + 0.4 * (l - g), 0.5 * (g + l), 0.16, 0.2, g + 0.7 * (l - g), 0.1])
    ux = np.array([0.0, 0.011, 0.004, -0.003, 0.002, -0.006, 0.0])
    uy = np.array([0.0, -0.004, 0.001, 0.002, -0.001, 0.003, 0.0])
    pxx = np.array([0, 1, -1, 1, -1, 0, 0, 0, 0], float)    # zero mass and momentum
    qx = np.array([0, -2, 0, 2, 0, 1, -1, -1, 1], float)     # zero mass and momentum
    f = np.zeros((9, ny, nx))
    for x in range(nx):
        fx = _feq(rho_x[x], ux[x], uy[x]) + 1e-3 * np.sin(x + 1.0) * pxx + 4e-4 * np.cos(2.0 * x) * qx
        f[:, :, x] = fx[:, None]
    fl = orc.fields(s, f)
    Fx, Fy = orc.force(s, f)
    out, _ = orc.step(s, f)
    for xb, xf, moving in ((0, 1, (1, 5, 8)), (nx - 1, nx - 2, (3, 6, 7))):
        rf = rho_x[xf]
        jx, jy = (f[:, 0, xf] * EX).sum(), (f[:, 0, xf] * EY).sum()
        vx, vy = jx / rf + Fx[0, xf] / (2 * rf), jy / rf + Fy[0, xf] / (2 * rf)
        rb = fl["rho"][0, xb]
        fstar = _feq(rb, vx, vy) + (1 - 1 / tau) * (f[:, 0, xf] - _feq(rf, vx, vy))
        # the column reports v_f as its velocity
        assert abs(fl["vx"][0, xb] - vx) <= 1e-15 and abs(fl["vy"][0, xb] - vy) <= 1e-15
        for i in moving:  # streamed one node into the lattice (uniform in y)
            assert abs(out[i, 0, xb + EX[i]] - fstar[i]) <= 2e-15 * abs(fstar[i]), (xb, i)
        for i in range(9):
            if EX[i] == EX[moving[0]]:  # slots fed from beyond the lattice's end: unchanged
                assert out[i, 0, xb] == f[i, 0, xb]
    assert abs(Fx[0, 1]) > 1e-4 and abs(Fx[0, nx - 2]) > 1e-4  # the velocity shift matters


def _wall_state(orc, rho, **kw):
    ny, nx = rho.shape
    s = orc.Setup(nx=nx, ny=ny, walls=True, **kw)
    return s, orc.init(s, rho)


@pytest.mark.parametrize("k", [1.0, 0.8])
def test_wall_pressure_kappa_terms_along_the_wall(orc, k):
    """rho = r0 + eps sin(q x) next to the wall: p_w - k^2 p0 tends to
    kappa rho q^2 eps sin(qx) - kappa/2 (q eps cos(qx))^2 at second order in q;
    where sin(qx) = 0 only the gradient term remains, where cos(qx) = 0 only
    the Laplacian term."""
    kappa, r0, eps, ny = 0.5, 0.12, 0.04, 9
    errs = []
    for nx in (48, 96, 192):
        q = 2 * np.pi / nx
        x = np.arange(nx)
        prof = r0 + eps * np.sin(q * x)
        s, f = _wall_state(orc, np.tile(prof, (ny, 1)), T_over_Tc=0.9, kappa=kappa, k=k)
        pf, _, _ = _eos_functions(s)
        pw = orc.fields(s, f)["p_wall"]
        rem = pw - k * k * np.array([pf(r) for r in prof])[None, :]
        lap_term = kappa * prof * q * q * eps * np.sin(q * x)
        grad_term = -0.5 * kappa * (q * eps * np.cos(q * x)) ** 2
        want = lap_term + grad_term
        assert np.abs(rem[0] - rem[1]).max() < 1e-17  # both walls alike
        errs.append(np.abs(rem[0] - want).max() / np.abs(lap_term).max())
        i0, i1 = 0, nx // 4  # sin = 0 (gradient term only) and cos = 0 (Laplacian only)
        assert abs(rem[0, i0] / grad_term[i0] - 1) < 0.02
        assert abs(rem[0, i1] / lap_term[i1] - 1) < 0.02
    assert errs[-1] < 2e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_wall_pressure_kappa_terms_across_the_wall(orc):
    """rho = r0 + eps cos(q (y - 1/2)) is even about both half-way wall planes, so
    the mirrored ghost rows continue it exactly: p_w - k^2 p0(rho_1) tends to
    -kappa rho_1 rho'' - kappa/2 rho'^2 at the first fluid row."""
    kappa, r0, eps = 0.5, 0.12, 0.04
    errs = []
    for h in (24, 48, 96):  # fluid rows; the wall planes are h apart
        ny = h + 2
        q = 2 * np.pi / h
        y = np.arange(ny)
        prof = r0 + eps * np.cos(q * (y - 0.5))
        s, f = _wall_state(orc, np.tile(prof[:, None], (1, 8)), T_over_Tc=0.9, kappa=kappa)
        pf, _, _ = _eos_functions(s)
        pw = orc.fields(s, f)["p_wall"]
        r1 = prof[1]
        d1 = -q * eps * np.sin(q * 0.5)       # rho'(y = 1)
        d2 = -q * q * eps * np.cos(q * 0.5)   # rho''(y = 1)
        want = -kappa * r1 * d2 - 0.5 * kappa * d1 * d1
        rem = pw[0, 0] - pf(r1)
        errs.append(abs(rem / want - 1))
        assert abs(pw[1, 3] - pw[0, 3]) < 1e-17
    assert errs[-1] < 1e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


@pytest.mark.parametrize("wet", [0.004, -0.003])
def test_wetting_offset_forces_of_a_uniform_liquid(orc, wet):
    """Uniform density r0 between walls, ghost rows r0 + wet at depths 1 and 2
    (R7). The D2Q9 stencils then give, exactly: lap rho = wet at the first fluid
    row, -wet on the first ghost row, 0 beyond; hence
      F_y(row 1)    = (phi(r0 + wet) - phi(r0)) / 2 + kappa r0 wet / 2,
      F_y(row 2)    = -kappa r0 wet / 2,   F_y(row 3) = 0,
    mirrored (sign flipped) at the top wall, F_x = 0 everywhere."""
    kappa, k, r0, nx, ny = 0.5, 0.9, 0.2, 6, 12
    s, f = _wall_state(orc, np.full((ny, nx), r0), T_over_Tc=0.85, kappa=kappa, k=k, wet=wet)
    pf, _, _ = _eos_functions(s)

    def phi(r):
        return k * k * pf(r) - r / 3

    Fx, Fy = orc.force(s, f)
    f1 = (phi(r0 + wet) - phi(r0)) / 2 + kappa * r0 * wet / 2
    f2 = -kappa * r0 * wet / 2
    assert np.abs(Fx).max() < 1e-17
    assert np.abs(Fy[1] - f1).max() <= 1e-13 * abs(f1)
    assert np.abs(Fy[2] - f2).max() <= 1e-13 * abs(f2)
    assert np.abs(Fy[3:ny - 3]).max() < 1e-17
    assert np.abs(Fy[ny - 2] + f1).max() <= 1e-13 * abs(f1)
    assert np.abs(Fy[ny - 3] + f2).max() <= 1e-13 * abs(f2)


def _contact_angle(orc, wet):
    nx, ny = 128, 64
    s = orc.Setup(nx=nx, ny=ny, walls=True, T_over_Tc=0.8, kappa=0.5, wet=wet)
    g, l, _ = s.coexistence()
    f = orc.init(s, synth.disk_rho0(nx, ny, 22, l, g, centre=(nx / 2, 0.5)))
    f, _ = orc.run(s, f, 6000)
    r = orc.fields(s, f)["rho"]
    mid = 0.5 * (r[1, nx // 2] + r[ny - 2, 0])
    col = r[1:ny - 1, nx // 2]
    i = int(np.argmax(col < mid))
    h = (i + (col[i - 1] - mid) / (col[i - 1] - col[i])) - 0.5
    row = r[1, :]
    ins = np.where(row > mid)[0]
    xl = ins[0] - (row[ins[0]] - mid) / (row[ins[0]] - row[ins[0] - 1])
    xr = ins[-1] + (row[ins[-1]] - mid) / (row[ins[-1]] - row[ins[-1] + 1])
    return 2 * np.degrees(np.arctan(h / (0.5 * (xr - xl))))


def test_wetting_offset_moves_the_contact_angle_both_ways(orc):
    """A denser ghost (wet > 0) makes the wall attract liquid: the sessile drop
    spreads below 90 degrees (about 80 at wet = 0.01); a lighter ghost (wet < 0)
    makes it bead up above 90 degrees (about 95 at wet = -0.005). Neutral
    wetting, wet = 0, is pinned at 90 +- 3 degrees."""
    hydrophilic = _contact_angle(orc, 0.01)
    hydrophobic = _contact_angle(orc, -0.005)
    assert hydrophilic < 86.0 and hydrophobic > 92.0, (hydrophilic, hydrophobic)

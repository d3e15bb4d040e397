"""Pins of the oracle's equation-of-state layer against independent routes.

The oracle solves the Carnahan-Starling critical point and the Maxwell
equal-area construction with its own bisections (chemical-potential form).
These tests re-derive the same quantities with sympy (symbolic derivatives,
nsolve) and scipy (equal-area integral in specific volume, brentq, quad), so
a wrong derivative, a wrong branch or a mis-scaled constant fails here.
"""
import math

import numpy as np
import pytest

sympy = pytest.importorskip("sympy")
scipy_opt = pytest.importorskip("scipy.optimize")
scipy_int = pytest.importorskip("scipy.integrate")

A, B, R = 1.0, 4.0, 1.0


def _cs_sym():
    rho, T = sympy.symbols("rho T", positive=True)
    eta = B * rho / 4
    p = rho * R * T * (1 + eta + eta**2 - eta**3) / (1 - eta) ** 3 - A * rho**2
    return rho, T, p


def test_critical_point_matches_sympy(orc):
    rho, T, p = _cs_sym()
    d1, d2 = sympy.diff(p, rho), sympy.diff(p, rho, 2)
    sol = sympy.nsolve([d1, d2], [rho, T], [0.13, 0.094], prec=30)
    Tc, rhoc = orc.cs_critical(A, B, R)
    assert abs(Tc - float(sol[1])) < 1e-13 * Tc
    assert abs(rhoc - float(sol[0])) < 1e-9 * rhoc


@pytest.mark.parametrize("t", [0.6, 0.8, 0.85, 0.95])
def test_p0_and_derivative_match_sympy(orc, t):
    rho, T, p = _cs_sym()
    Tc, _ = orc.cs_critical()
    Tv = t * Tc
    pf = sympy.lambdify(rho, p.subs(T, Tv))
    dpf = sympy.lambdify(rho, sympy.diff(p, rho).subs(T, Tv))
    for r in np.linspace(0.005, 0.6, 23):
        assert abs(orc.cs_p0(A, B, R, Tv, r) - pf(r)) < 1e-14 * max(1.0, abs(pf(r)))
        assert abs(orc.cs_dp0(A, B, R, Tv, r) - dpf(r)) < 1e-12 * max(1.0, abs(dpf(r)))


def test_chemical_potential_is_integral_of_dp_over_rho(orc):
    """Gibbs-Duhem at fixed T: d mu = dp0 / rho (Eq. 2.5 differentiated)."""
    Tc, _ = orc.cs_critical()
    Tv = 0.8 * Tc
    for r1, r2 in [(0.01, 0.05), (0.02, 0.3), (0.1, 0.4)]:
        val, _ = scipy_int.quad(lambda r: orc.cs_dp0(A, B, R, Tv, r) / r, r1, r2,
                                epsabs=1e-14, epsrel=1e-13)
        dmu = orc.cs_mu(A, B, R, Tv, r2) - orc.cs_mu(A, B, R, Tv, r1)
        assert abs(dmu - val) < 1e-11 * max(1.0, abs(val))


def _maxwell_scipy(Tv):
    """Equal-area rule in specific volume v = 1/rho: int_{v_l}^{v_g} p dv = p_sat (v_g - v_l)."""
    rho, T, p = _cs_sym()
    pf = sympy.lambdify(rho, p.subs(T, Tv))
    dpf = sympy.lambdify(rho, sympy.diff(p, rho).subs(T, Tv))
    rc = 0.1304438842
    s1 = scipy_opt.brentq(dpf, 1e-6, rc, xtol=1e-15)
    s2 = scipy_opt.brentq(dpf, rc, 0.99, xtol=1e-15)

    def roots(ps):
        rg = scipy_opt.brentq(lambda r: pf(r) - ps, 1e-12, s1, xtol=1e-16)
        rl = scipy_opt.brentq(lambda r: pf(r) - ps, s2, 0.999, xtol=1e-16)
        return rg, rl

    def area(ps):
        rg, rl = roots(ps)
        integral, _ = scipy_int.quad(lambda v: pf(1.0 / v), 1.0 / rl, 1.0 / rg,
                                     epsabs=1e-15, epsrel=1e-13, limit=200)
        return integral - ps * (1.0 / rg - 1.0 / rl)

    lo = max(pf(s2), 1e-12) * (1 + 1e-9)
    hi = pf(s1) * (1 - 1e-9)
    ps = scipy_opt.brentq(area, lo, hi, xtol=1e-16, rtol=1e-14)
    rg, rl = roots(ps)
    return rg, rl, ps


@pytest.mark.parametrize("t", [0.7, 0.8, 0.85, 0.95])
def test_maxwell_matches_equal_area_in_specific_volume(orc, t):
    Tc, _ = orc.cs_critical()
    g, l, p = orc.maxwell(A, B, R, t * Tc)
    g2, l2, p2 = _maxwell_scipy(t * Tc)
    assert abs(g - g2) < 1e-8 * g2
    assert abs(l - l2) < 1e-9 * l2
    assert abs(p - p2) < 1e-8 * p2
    # equal pressure on both branches
    assert abs(orc.cs_p0(A, B, R, t * Tc, g) - p) < 1e-12 * p
    assert abs(orc.cs_p0(A, B, R, t * Tc, l) - p) < 1e-10 * p


def test_maxwell_rejects_supercritical(orc):
    Tc, _ = orc.cs_critical()
    with pytest.raises(ValueError):
        orc.maxwell(A, B, R, 1.01 * Tc)


def test_gas_root_inverts_eos_on_gas_branch(orc):
    Tc, _ = orc.cs_critical()
    Tv = 0.85 * Tc
    g, l, psat = orc.maxwell(A, B, R, Tv)
    for target in (0.5 * psat, psat, psat + 5e-4, psat - 5e-4):
        r = orc.gas_root(A, B, R, Tv, target)
        assert abs(orc.cs_p0(A, B, R, Tv, r) - target) < 1e-13
        assert orc.cs_dp0(A, B, R, Tv, r) > 0.0     # stable (gas) branch
        assert r < l
    assert math.isclose(orc.gas_root(A, B, R, Tv, psat), g, rel_tol=1e-9)
    with pytest.raises(ValueError):
        orc.gas_root(A, B, R, Tv, 10 * psat)  # above the gas spinodal pressure

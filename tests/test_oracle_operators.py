"""Pins of the oracle's lattice operators: equilibrium, stencils and force.

Independent routes: closed-form moments of the equilibrium (Eq. 2.2), exactness
of the discrete gradient / Laplacian on polynomials and their continuum limit
(Taylor expansion, isotropic O(q^2) error), telescoping sums, and the
continuum form of the force of Eq. 2.17 on long-wavelength profiles, where
derivatives are taken analytically.
"""
import numpy as np
import pytest

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (0.3, 0.05, -0.02), (0.02, -0.1, 0.07)])
def test_equilibrium_moments(orc, rho, ux, uy):
    f = orc.feq(rho, ux, uy)
    assert abs(f.sum() - rho) < 1e-15
    assert abs((f * EX).sum() - rho * ux) < 1e-16
    assert abs((f * EY).sum() - rho * uy) < 1e-16
    # second moments: rho/3 I + rho u u
    assert abs((f * EX * EX).sum() - (rho / 3 + rho * ux * ux)) < 1e-15
    assert abs((f * EY * EY).sum() - (rho / 3 + rho * uy * uy)) < 1e-15
    assert abs((f * EX * EY).sum() - rho * ux * uy) < 1e-16


def test_stencils_exact_on_quadratics(orc):
    ny, nx = 40, 48
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    c = [0.3, -0.7, 1.1, 0.25, -0.4, 0.6]  # c0 + c1 x + c2 y + c3 x^2 + c4 xy + c5 y^2
    psi = c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y
    gx, gy = orc.grad_periodic(psi)
    lap = orc.lap_periodic(psi)
    inner = (slice(2, ny - 2), slice(2, nx - 2))  # away from the periodic seam
    assert np.abs(gx[inner] - (c[1] + 2 * c[3] * x + c[4] * y)[inner]).max() < 1e-11
    assert np.abs(gy[inner] - (c[2] + c[4] * x + 2 * c[5] * y)[inner]).max() < 1e-11
    assert np.abs(lap[inner] - (2 * c[3] + 2 * c[5])).max() < 1e-11


@pytest.mark.parametrize("theta", [0.0, 0.3, np.pi / 4, 1.1])
def test_laplacian_continuum_limit_isotropic(orc, theta):
    """On sin(q.x) the discrete Laplacian approaches -|q|^2 with an isotropic
    relative error q^2/12 (the nine-point stencil's known leading term)."""
    n = 256
    errs = []
    for m in (4, 8):
        # wave vector commensurate with the periodic box along both axes
        qx = 2 * np.pi * round(m * np.cos(theta)) / n
        qy = 2 * np.pi * round(m * np.sin(theta)) / n
        q2 = qx * qx + qy * qy
        y, x = np.mgrid[0:n, 0:n].astype(float)
        psi = np.sin(qx * x + qy * y)
        lap = orc.lap_periodic(psi)
        ratio = (lap * psi).sum() / (psi * psi).sum()  # Rayleigh quotient = symbol
        errs.append((ratio + q2) / q2 - q2 / 12.0)
        assert abs(ratio + q2) < 0.01 * q2
    # remaining error is O(q^4): grows ~16x when q doubles (m = 4 -> 8)
    assert abs(errs[0]) < abs(errs[1]) / 8 + 1e-12


def test_gradient_telescopes_on_periodic_box(orc):
    rng = np.random.default_rng(5)
    psi = rng.standard_normal((33, 47))
    gx, gy = orc.grad_periodic(psi)
    assert abs(gx.sum()) < 1e-11 and abs(gy.sum()) < 1e-11
    assert abs(orc.lap_periodic(psi).sum()) < 1e-11


def _state_from_rho(orc, setup, rho):
    return orc.init(setup, rho)


def test_force_vanishes_on_uniform_density(orc):
    s = orc.Setup(nx=16, ny=12, T_over_Tc=0.8, kappa=0.5)
    f = _state_from_rho(orc, s, np.full((12, 16), 0.17))
    Fx, Fy = orc.force(s, f)
    assert np.abs(Fx).max() < 1e-17 and np.abs(Fy).max() < 1e-17


def test_force_adds_uniform_body_force(orc):
    s = orc.Setup(nx=16, ny=12, T_over_Tc=0.8, kappa=0.5, gx=3e-6, gy=-2e-6)
    f = _state_from_rho(orc, s, np.full((12, 16), 0.17))
    Fx, Fy = orc.force(s, f)
    assert np.allclose(Fx, 3e-6, rtol=0, atol=1e-18) and np.allclose(Fy, -2e-6, rtol=0, atol=1e-18)


@pytest.mark.parametrize("k,kappa", [(1.0, 0.5), (0.5, 0.5), (1.0, 0.0), (0.7, 2.0)])
def test_force_continuum_limit(orc, k, kappa):
    """Eq. 2.17 in the mesh space: F = -grad(k^2 p0 - rho/3) + kappa rho grad(lap rho).
    On rho = r0 + e sin(q y) the exact continuum force is
    F_y = -(k^2 p0'(rho) - 1/3) rho' + kappa rho rho''' with rho' = e q cos, rho''' = -e q^3 cos;
    the discrete force must approach it with an O(q^2) relative error."""
    n = 128
    rel = []
    for m in (2, 4):
        s = orc.Setup(nx=4, ny=n, T_over_Tc=0.9, k=k, kappa=kappa)
        q = 2 * np.pi * m / n
        e = 1e-3
        y = np.arange(n, dtype=float)
        r = 0.2 + e * np.sin(q * y)
        f = _state_from_rho(orc, s, np.repeat(r[:, None], 4, axis=1))
        Fx, Fy = orc.force(s, f)
        dp = np.array([orc.cs_dp0(s.a, s.b, s.R, s.T, v) for v in r])
        r1 = e * q * np.cos(q * y)
        r3 = -e * q ** 3 * np.cos(q * y)
        exact = -(k * k * dp - 1.0 / 3.0) * r1 + kappa * r * r3
        err = np.abs(Fy[:, 0] - exact).max() / np.abs(exact).max()
        rel.append(err)
        assert np.abs(Fx).max() < 1e-16
        assert err < 0.15
    assert rel[0] < rel[1] / 3  # second-order convergence in q


def test_force_is_affine_in_k_squared(orc):
    rng = np.random.default_rng(2)
    rho = 0.15 + 0.05 * rng.random((20, 24))
    F = []
    for k in (0.5, 1.0, 1.5):
        s = orc.Setup(nx=24, ny=20, T_over_Tc=0.8, k=k, kappa=0.3)
        F.append(orc.force(s, _state_from_rho(orc, s, rho))[0])
    # F(k) = A k^2 + B  ->  second difference in k^2 vanishes
    k2 = np.array([0.25, 1.0, 2.25])
    slope1 = (F[1] - F[0]) / (k2[1] - k2[0])
    slope2 = (F[2] - F[1]) / (k2[2] - k2[1])
    assert np.abs(slope1 - slope2).max() < 1e-13

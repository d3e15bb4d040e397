"""Pins of the oracle's general wall geometry (a per-node solid mask).

The paper's airway is a straight channel (Sec. 2.2); a mask generalises its
walls to any solid nodes: half-way bounce-back on every link into a solid
node, and ghost densities of solid points from the mirror rule generalised
(axis directions of least depth, else diagonals, else knight offsets; plus
the wetting offset). Each check compares against something the mask code does
not compute itself: the channel rule of the wall rows, the same channel
turned by 90 degrees, conservation of mass, invariance of a resting uniform
state, the mirror symmetry of a symmetric geometry, and the 90-degree contact
angle of neutral wetting on an obstacle's face.
"""
import numpy as np
import pytest

import synth

# D2Q9 directions under the transposition x <-> y: 1 (1,0) <-> 2 (0,1),
# 3 <-> 4, 5 <-> 5, 6 (-1,1) <-> 8 (1,-1), 7 <-> 7
TRANSPOSE = [0, 2, 1, 4, 3, 5, 8, 7, 6]
MIRROR_Y = [0, 1, 4, 3, 2, 8, 7, 6, 5]  # y -> -y


def test_empty_mask_is_the_channel_rule(orc):
    """A mask with no solid node beyond the wall rows runs the general ghost
    rule, which on flat walls must reproduce the channel's mirror rule bit for
    bit (wetting offset included), as must bounce-back and the diagnostics."""
    nx, ny = 96, 40
    for kw in (dict(walls=True, bc_x=True, dp=4e-4, wet=0.01), dict(walls=True, bc_x=False, wet=-0.004, gx=2e-6)):
        s0 = orc.Setup(nx=nx, ny=ny, T_over_Tc=0.85, kappa=0.5, **kw)
        m = np.zeros((ny, nx), np.uint8)
        m[0] = m[-1] = 1  # the wall rows are solid either way
        s1 = orc.Setup(nx=nx, ny=ny, T_over_Tc=0.85, kappa=0.5, mask=m, **kw)
        g, l, _ = s0.coexistence()
        f = orc.init(s0, synth.airway_rho0(nx, ny, 5, 30, 20, l, g, noise=1e-3, seed=3))
        a, da = orc.run(s0, f, 150)
        b, db = orc.run(s1, f, 150)
        assert np.array_equal(a, b)
        assert da == db


def _h_channel(orc, nx, H, **kw):
    ny = H + 2
    s = orc.Setup(nx=nx, ny=ny, walls=True, T_over_Tc=0.85, kappa=0.5, **kw)
    g, l, _ = s.coexistence()
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    rho = synth.airway_rho0(nx, ny, 4, 10, 12, l, g) + 0.01 * np.sin(2 * np.pi * x / nx) * np.cos(y)
    return s, rho


def test_mask_walls_equal_the_channel_turned_by_90_degrees(orc):
    """The channel with solid rows, against the same channel standing upright
    in a periodic box whose walls are three mask columns per side: the fields
    agree node for node (to rounding: the stencil sums run over the directions
    in another order), with x and y exchanged."""
    nx, H = 48, 20
    gx = 3e-6
    s, rho = _h_channel(orc, nx, H, gx=gx, wet=0.003)
    f = orc.init(s, rho)
    a, _ = orc.run(s, f, 300)
    fa = orc.fields(s, a)
    # upright copy: column x' = y + 2 holds row y; three solid columns per side
    W = H + 6
    m = np.zeros((nx, W), np.uint8)
    m[:, :3] = m[:, -3:] = 1
    s2 = orc.Setup(nx=W, ny=nx, T_over_Tc=0.85, kappa=0.5, gy=gx, wet=0.003, mask=m)
    rho2 = np.full((nx, W), rho.mean())
    rho2[:, 2:H + 4] = rho.T  # rows 0..H+1 of the channel (wall rows are solid in both)
    f2 = orc.init(s2, rho2)
    b, _ = orc.run(s2, f2, 300)
    fb = orc.fields(s2, b)
    ra = fa["rho"][1:H + 1, :]
    rb = fb["rho"][:, 3:H + 3].T
    assert np.abs(ra - rb).max() <= 1e-12 * ra.max()
    vscale = np.abs(fa["vx"]).max()
    assert vscale > 1e-5
    assert np.abs(fa["vx"][1:H + 1, :] - fb["vy"][:, 3:H + 3].T).max() <= 1e-9 * vscale
    assert np.abs(fa["vy"][1:H + 1, :] - fb["vx"][:, 3:H + 3].T).max() <= 1e-9 * vscale
    # the populations themselves, directions exchanged
    pa = a[:, 1:H + 1, :]
    pb = np.stack([b[TRANSPOSE[i]][:, 3:H + 3].T for i in range(9)])
    assert np.abs(pa - pb).max() <= 1e-12 * pa.max()


def _obstacle_mask(nx, ny):
    m = np.zeros((ny, nx), np.uint8)
    m[1:12, 40:56] = 1                        # a block on the bottom wall
    yy, xx = np.mgrid[0:ny, 0:nx]
    m[(xx - 72) ** 2 + (yy - 30) ** 2 <= 25] = 1  # a free disk
    m[0] = m[-1] = 1
    return m


def test_obstacles_conserve_mass_and_rest(orc):
    nx, ny = 96, 48
    m = _obstacle_mask(nx, ny)
    # a uniform state at rest stays exactly at rest under neutral wetting
    # (uniform ghosts, symmetric bounce-back)
    rest = orc.Setup(nx=nx, ny=ny, walls=True, T_over_Tc=0.8, kappa=0.5, mask=m)
    f = orc.init(rest, np.full((ny, nx), 0.2))
    g1, _ = orc.run(rest, f, 40)
    fluid = m == 0
    assert np.abs(g1[:, fluid] - f[:, fluid]).max() < 1e-15
    # a two-phase state next to both obstacles, wetting offset on: mass to 1e-12
    s = orc.Setup(nx=nx, ny=ny, walls=True, T_over_Tc=0.8, kappa=0.5, wet=0.005, mask=m)
    g, l, _ = s.coexistence()
    rho0 = synth.disk_rho0(nx, ny, 14, l, g, noise=1e-3, seed=9, centre=(60.0, 24.0))
    f = orc.init(s, rho0)
    _, d0 = orc.step(s, f)
    f, _ = orc.run(s, f, 3000)
    _, d1 = orc.step(s, f)
    assert abs(d1["mass"] / d0["mass"] - 1) <= 1e-12
    r = orc.fields(s, f)["rho"]
    assert (r[m == 1] == 0).all() and (r[fluid] > 0).all()


def test_symmetric_geometry_keeps_its_mirror_symmetry(orc):
    """A cross-shaped obstacle (its inner corners take the diagonal rule) on the
    centre line of a channel, a two-phase state and a body force along x, all
    mirror-symmetric about the centre line: the flow must stay symmetric (rho
    and v_x even, v_y odd) and the populations mirror with e_y -> -e_y."""
    nx, ny = 80, 42  # fluid rows 1..40, mirror y <-> 41 - y
    m = np.zeros((ny, nx), np.uint8)
    m[0] = m[-1] = 1
    m[15:27, 36:40] = 1   # cross: vertical bar
    m[19:23, 30:46] = 1   # horizontal bar
    assert np.array_equal(m, m[::-1])
    s = orc.Setup(nx=nx, ny=ny, walls=True, T_over_Tc=0.8, kappa=0.5, gx=2e-6, wet=0.004, mask=m)
    g, l, _ = s.coexistence()
    rho0 = synth.airway_rho0(nx, ny, 4, 55, 10, l, g)
    rho0 = 0.5 * (rho0 + rho0[::-1])
    assert np.array_equal(rho0, rho0[::-1])
    f = orc.init(s, rho0)
    f, _ = orc.run(s, f, 400)
    fl = orc.fields(s, f)
    r = fl["rho"]
    assert np.abs(r - r[::-1]).max() <= 1e-12 * r.max()
    vs = np.abs(fl["vx"]).max()
    assert vs > 1e-6
    assert np.abs(fl["vx"] - fl["vx"][::-1]).max() <= 1e-9 * vs
    assert np.abs(fl["vy"] + fl["vy"][::-1]).max() <= 1e-9 * vs
    fm = np.stack([f[MIRROR_Y[i]][::-1] for i in range(9)])
    fluid = m == 0
    assert np.abs(f[:, fluid] - fm[:, fluid]).max() <= 1e-12 * f.max()


def test_geometry_symmetric_under_transposition_stays_symmetric(orc):
    """A plus-shaped obstacle in a periodic square box, droplets on the diagonal
    and a body force along it: the state is symmetric under x <-> y and must
    stay so. A ghost rule that favoured one axis where two are equally deep
    (the plus's inner corners) would break this symmetry."""
    n = 64
    m = np.zeros((n, n), np.uint8)
    m[22:42, 30:34] = 1
    m[30:34, 22:42] = 1
    assert np.array_equal(m, m.T)
    s = orc.Setup(nx=n, ny=n, T_over_Tc=0.8, kappa=0.5, gx=1e-6, gy=1e-6, wet=0.004, mask=m)
    g, l, _ = s.coexistence()
    rho0 = np.maximum(synth.disk_rho0(n, n, 8, l, g, centre=(14.0, 14.0)),
                      synth.disk_rho0(n, n, 8, l, g, centre=(50.0, 50.0)))
    assert np.array_equal(rho0, rho0.T)
    f = orc.init(s, rho0)
    f, _ = orc.run(s, f, 400)
    fl = orc.fields(s, f)
    r = fl["rho"]
    assert np.abs(r - r.T).max() <= 1e-12 * r.max()
    vs = np.abs(fl["vx"]).max()
    assert vs > 1e-6
    assert np.abs(fl["vx"] - fl["vy"].T).max() <= 1e-9 * vs


def _angle_on_block(orc, wet):
    nx, ny = 128, 72
    top = 16  # block rows 1..15, its face is the half-way plane y = 15.5
    m = np.zeros((ny, nx), np.uint8)
    m[0] = m[-1] = 1
    m[1:top, 20:108] = 1
    s = orc.Setup(nx=nx, ny=ny, walls=True, T_over_Tc=0.8, kappa=0.5, wet=wet, mask=m)
    g, l, _ = s.coexistence()
    rho0 = synth.disk_rho0(nx, ny, 20, l, g, centre=(nx / 2, top - 0.5))
    rho0[m == 1] = g
    f = orc.init(s, rho0)
    f, _ = orc.run(s, f, 6000)
    r = orc.fields(s, f)["rho"]
    mid = 0.5 * (r[top, nx // 2] + r[ny - 2, 2])
    col = r[top:ny - 1, nx // 2]
    i = int(np.argmax(col < mid))
    h = (i + (col[i - 1] - mid) / (col[i - 1] - col[i])) + 0.5  # from the face plane top - 0.5
    row = r[top, :]
    ins = np.where(row > mid)[0]
    xl = ins[0] - (row[ins[0]] - mid) / (row[ins[0]] - row[ins[0] - 1])
    xr = ins[-1] + (row[ins[-1]] - mid) / (row[ins[-1]] - row[ins[-1] + 1])
    assert 20 < xl and xr < 108  # the contact line sits on the face, away from its edges
    return 2 * np.degrees(np.arctan(h / (0.5 * (xr - xl))))


def test_contact_angle_on_an_obstacle_face(orc):
    """Neutral wetting (wet = 0) on the flat top face of a block: 90 +- 4
    degrees; a positive offset makes the face hydrophilic (below 86)."""
    assert abs(_angle_on_block(orc, 0.0) - 90.0) < 4.0
    assert _angle_on_block(orc, 0.01) < 86.0

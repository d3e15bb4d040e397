"""The slot algebra of in-place (AA pattern) streaming, on the CPU.

The in-place step reads and writes one array: even steps read a node's own
slots F[x][i] and write f*_i to F[x][opp(i)]; odd steps read f_i(x) from
F[x - e_i][opp(i)] and write f*_i to F[x + e_i][i]; half-way bounce-back
writes into the wall row's slot F[x + e_i][i] on even steps and into
F[x][opp(i)] on odd steps; the layout swap trades (x, i) and (x - e_i,
opp(i)). These rules, emulated here with an identity collision (f* = f, so
only the data movement is exercised), must reproduce plain two-array push
streaming with bounce-back step after step, touch every slot at most once per
step, never write a slot that another node reads in the same step, and return
to the natural layout after an even number of steps or one swap. A dropped
reversal, a wrong shift sign or a bounce into the wrong slot fails one of them.
"""
import numpy as np
import pytest

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])


def _push(f, walls):
    """Two-array streaming: g[i](x + e_i) = f[i](x), bounce-back off rows 0 and ny-1."""
    _, ny, nx = f.shape
    g = f.copy()
    ys = range(1, ny - 1) if walls else range(ny)
    for y in ys:
        for x in range(nx):
            for i in range(9):
                ty, tx = y + EY[i], (x + EX[i]) % nx
                if walls and (ty == 0 or ty == ny - 1):
                    g[OPP[i], y, x] = f[i, y, x]
                else:
                    g[i, ty % ny, tx] = f[i, y, x]
    return g


def _aa_step(F, walls, odd):
    """One in-place step; returns {slot: reading node} and {slot: writing node}."""
    _, ny, nx = F.shape
    ys = range(1, ny - 1) if walls else range(ny)
    reader, writer = {}, {}
    for y in ys:
        for x in range(nx):
            src = []
            for i in range(9):
                s = ((OPP[i], (y - EY[i]) % ny, (x - EX[i]) % nx) if odd else (i, y, x))
                src.append(s)
            f = [F[s] for s in src]
            dst = []
            for i in range(9):
                ty, tx = y + EY[i], (x + EX[i]) % nx
                wall = walls and (ty == 0 or ty == ny - 1)
                if odd:
                    d = (OPP[i], y, x) if wall else (i, ty % ny, tx)
                else:
                    d = (i, ty, tx) if wall else (OPP[i], y, x)
                dst.append(d)
            for s in src:
                assert s not in reader
                reader[s] = (y, x)
            for d, v in zip(dst, f):
                assert d not in writer
                writer[d] = (y, x)
                F[d] = v
    return reader, writer


def _odd_view(F):
    """The logical state held by an odd-parity array: f_i(x) = F[x - e_i][opp(i)]."""
    _, ny, nx = F.shape
    f = np.empty_like(F)
    for i in range(9):
        f[i] = np.roll(np.roll(F[OPP[i]], EY[i], axis=0), EX[i], axis=1)
    return f


def _swap(F, walls):
    _, ny, nx = F.shape
    G = F.copy()
    for y in range(ny):
        for x in range(nx):
            for i in (1, 2, 5, 6):
                sy, sx = y - EY[i], (x - EX[i]) % nx
                if walls and not (0 <= sy < ny):
                    continue
                a, b = (i, y, x), (OPP[i], sy % ny, sx)
                G[a], G[b] = F[b], F[a]
    return G


@pytest.mark.parametrize("nx,ny,walls", [(7, 6, True), (5, 4, True), (6, 5, False), (1, 5, False), (3, 1, False)])
def test_aa_rules_reproduce_push_streaming(nx, ny, walls):
    rng = np.random.default_rng(nx * 10 + ny)
    f = rng.random((9, ny, nx))
    F = f.copy()
    fluid = slice(1, ny - 1) if walls else slice(0, ny)
    ref = f
    for step in range(6):
        odd = step % 2 == 1
        reader, writer = _aa_step(F, walls, odd)
        # no slot is read by one node and written by another in the same step
        # (bounce-back writes into wall-row slots no fluid node reads)
        for slot, node in writer.items():
            assert reader.get(slot, node) == node, (step, slot)
        ref = _push(ref, walls)
        state = _odd_view(F) if not odd else F  # after an even step the array holds the odd layout
        assert np.array_equal(state[:, fluid], ref[:, fluid]), step
        if not odd:
            # the layout swap turns the odd-parity array into the natural one
            assert np.array_equal(_swap(F, walls)[:, fluid], ref[:, fluid]), step


def test_swap_is_an_involution_on_stored_slots():
    rng = np.random.default_rng(5)
    for walls in (True, False):
        F = rng.random((9, 6, 7))
        assert np.array_equal(_swap(_swap(F, walls), walls), F)

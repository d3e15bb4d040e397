"""Seeded synthetic inputs shared by the tests, the oracle runs and the benchmark.

This module holds no arithmetic of the lattice Boltzmann method: it only builds
initial density fields (smooth tanh profiles of a disk, a wall film and a
liquid plug, plus optional uniform noise) and draws the parameters of a
batched sweep. Coexistence densities are inputs here; each side computes its
own from the equation of state.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based hash:
the draw for node index n under seed s is splitmix64(s ^ n), whose top 53 bits
give u in [0, 1). The product library implements the same published
generator in its host helper; neither copy calls the other.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied to x (uint64 array), all arithmetic mod 2^64."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, idx: np.ndarray) -> np.ndarray:
    """u in [0, 1) for counter idx under seed: top 53 bits of splitmix64(seed ^ idx)."""
    z = splitmix64(np.uint64(seed) ^ np.asarray(idx, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def node_noise(nx: int, ny: int, amp: float, seed: int) -> np.ndarray:
    """amp * (2u - 1) per node, node index n = y * nx + x."""
    idx = np.arange(nx * ny, dtype=np.uint64).reshape(ny, nx)
    return amp * (2.0 * uniform01(seed, idx) - 1.0)


def disk_rho0(nx, ny, radius, rho_l, rho_g, width=4.0, noise=0.0, seed=1, centre=None):
    """Liquid disk of the given radius in vapour: S = (1 - tanh(2 (r - R0) / W)) / 2."""
    cx, cy = (nx / 2.0, ny / 2.0) if centre is None else centre
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    s = 0.5 * (1.0 - np.tanh(2.0 * (r - radius) / width))
    rho = rho_g + (rho_l - rho_g) * s
    if noise:
        rho = rho + node_noise(nx, ny, noise, seed)
    return rho


def slab_rho0(nx, ny, y_lo, y_hi, rho_l, rho_g, width=4.0):
    """Flat liquid slab between rows y_lo and y_hi (periodic box)."""
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    s = 0.5 * (np.tanh(2.0 * (y - y_lo) / width) - np.tanh(2.0 * (y - y_hi) / width))
    return rho_g + (rho_l - rho_g) * s


def airway_rho0(nx, ny, film, plug_x, plug_len, rho_l, rho_g, width=4.0, noise=0.0, seed=1):
    """Channel with solid rows 0 and ny-1: a wall film of thickness `film` (distance
    from the half-way wall plane) and a liquid plug spanning x in [plug_x, plug_x + plug_len).
    S = max(s_film, s_plug); both profiles are smooth in film and plug_len."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d_wall = np.minimum(y - 0.5, (ny - 1.5) - y)
    s_film = 0.5 * (1.0 - np.tanh(2.0 * (d_wall - film) / width))
    s_plug = 0.5 * (np.tanh(2.0 * (x - plug_x) / width)
                    - np.tanh(2.0 * (x - plug_x - plug_len) / width))
    s = np.maximum(s_film, s_plug)
    rho = rho_g + (rho_l - rho_g) * s
    if noise:
        rho = rho + node_noise(nx, ny, noise, seed)
    return rho


def sweep_channels(n=64, seed=3):
    """Per-channel sizes and parameters of the batched parameter sweep:
    height in [128, 512], length in [1024, 4096], pressure drop in [5e-4, 3e-3],
    plug length in [64, 256] at x = length / 4, film thickness in [4, 24]."""
    out = []
    for c in range(n):
        u = uniform01(seed, np.arange(5, dtype=np.uint64) + np.uint64(5 * c))
        h = 128 + int(u[0] * (512 - 128 + 1))
        length = 1024 + int(u[1] * (4096 - 1024 + 1))
        out.append({
            "ny": h,
            "nx": length,
            "dp": 5e-4 + u[2] * (3e-3 - 5e-4),
            "plug_len": 64 + int(u[3] * (256 - 64 + 1)),
            "plug_x": length // 4,
            "film": 4 + int(u[4] * (24 - 4 + 1)),
        })
    return out

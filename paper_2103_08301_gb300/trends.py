"""Plug rupture and the wall-load trends of the parameter study (Sec. 3.3, Figs. 10-12).

The paper drives the liquid plug with a body force F along the airway, the
ends extrapolated at one pressure (Sec. 2.2), and reports per run the rupture,
the aerosol (droplets detached from the wall films) and the differences
between the maximum and the minimum of the wall pressure P_wall and of the
wall shear stress tau_wall, against F, the plug length b and the film
thickness h. This module runs such a channel through the C ABI:

  - the operating point is the method's own coexistence
    (lbm_relaxed_coexistence): both ends at its saturation pressure p*, the
    initial wall films and plug at its liquid density in its vapour;
  - the step kernels accumulate the wall-load extrema of every step; the
    accumulators are restarted after `settle` steps, so the initial relaxation
    of the tanh profiles does not count;
  - every `every` steps the density is read back and lbm_plug_analysis gives
    the plug ends, whether the plug still closes the channel and the detached
    droplets; the rupture is the first such read-back at which the plug no
    longer closes the channel while its front had not reached the outlet;
    the run stops `window` steps after it (the reopened channel's vapour is
    then driven freely by the body force).

Only host orchestration lives here: every step runs in the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np

from . import Lattice, lbm_airway_rho0, lbm_eos, lbm_plug_analysis, lbm_relaxed_coexistence


def method_coexistence(T_over_Tc=0.85, k=1.0, kappa=0.5, tau=1.0, stream=None):
    """(rho_g*, rho_l*, p*) of the method at these parameters (FP64 slab on the GPU)."""
    c = lbm_relaxed_coexistence(lbm_eos(1.0, 4.0, 1.0, T_over_Tc, k, kappa), tau, None, 64, 192, 40000,
                                stream=stream)
    return c["rho_g"], c["rho_l"], c["p_gas"]


def rupture_run(nx, ny, film, plug_len, force, *, plug_x=None, precision=32, T_over_Tc=0.85, k=1.0,
                kappa=0.5, tau=1.0, coex=None, settle=2000, every=500, window=3000, max_steps=200000,
                stream=None):
    """One airway channel under a body force until the plug ruptures.

    Returns dict(rupture_step (None if none within max_steps), steps, dP_wall,
    dtau_wall (max - min over the steps after `settle`), droplet_mass and
    n_droplets (the largest aerosol seen after the rupture), history (step,
    x_rear, x_front, intact, n_droplets, droplet_mass per read-back), nan).
    """
    rg, rl, ps = coex if coex is not None else method_coexistence(T_over_Tc, k, kappa, tau, stream)
    plug_x = nx // 5 if plug_x is None else plug_x
    rho0 = lbm_airway_rho0(nx, ny, film, plug_x, plug_len, rl, rg)
    mid = 0.5 * (rg + rl)
    out = {"rupture_step": None, "history": [], "droplet_mass": 0.0, "n_droplets": 0, "nan": False}
    with Lattice(nx, ny, rho0, walls=True, bc_x=True, precision=precision, T_over_Tc=T_over_Tc, k=k,
                 kappa=kappa, tau=tau, dp=0.0, p_ref=ps, gx=force, stream=stream) as lat:
        lat.step(settle)
        lat.reset_diag()
        step, front, stop_at = settle, plug_x + plug_len, max_steps
        while step < stop_at:
            n = min(every, stop_at - step)
            lat.step(n)
            step += n
            rho = lat.fields()["rho"].astype(np.float64)
            if not np.isfinite(rho).all():
                out["nan"] = True
                break
            st = lbm_plug_analysis(rho, mid)
            out["history"].append((step, st["x_rear"], st["x_front"], st["intact"], st["n_droplets"],
                                   st["droplet_mass"]))
            if out["rupture_step"] is None:
                if not st["intact"] and front < nx - 8:
                    out["rupture_step"] = step
                    stop_at = min(max_steps, step + window)
                elif not math.isnan(st["x_front"]):
                    front = st["x_front"]
            if out["rupture_step"] is not None and st["droplet_mass"] > out["droplet_mass"]:
                out["droplet_mass"], out["n_droplets"] = st["droplet_mass"], st["n_droplets"]
        d = lat.diag()
    out["steps"] = step
    out["dP_wall"] = d["p_wall_max"] - d["p_wall_min"]
    out["dtau_wall"] = d["tau_wall_max"] - d["tau_wall_min"]
    out["nan"] = out["nan"] or bool(d["nan_detected"])
    return out


def sweep(base, vary, **kw):
    """Rupture runs of `base` (dict nx, ny, film, plug_len, force) with one
    parameter changed at a time: vary = {name: [values]}. Returns a list of
    (name, value, result)."""
    coex = kw.pop("coex", None)
    if coex is None:
        coex = method_coexistence(kw.get("T_over_Tc", 0.85), kw.get("k", 1.0), kw.get("kappa", 0.5),
                                  kw.get("tau", 1.0), kw.get("stream"))
    rows = []
    for name, values in vary.items():
        for v in values:
            p = dict(base)
            p[name] = v
            rows.append((name, v, rupture_run(p["nx"], p["ny"], p["film"], p["plug_len"], p["force"], coex=coex,
                                              **kw)))
    return rows

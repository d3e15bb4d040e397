"""Gradients of time-integrated wall loads through the discrete adjoint.

Binding of the ``lbm_adjoint_*`` entry points of ``include/lbm.h`` plus two
``torch.autograd.Function`` wrappers:

- ``WallLoads``: (rho0, dp, gx, gy) -> (J_tau, J_p), the wall shear and wall
  pressure summed over the walls' interior columns and the states that
  ``nsteps`` steps read (Sec. 3, Figs. 10-12). Its backward runs the adjoint
  kernels of ``liblbm.so`` (checkpoint-and-recompute over blocks of steps).
- ``AirwayProfile``: (film, plug_len) -> rho0, the initial airway density of
  ``lbm_airway_rho0``, with its exact tangent from ``lbm_airway_rho0_tangent``.

Chained, they give dJ/d(pressure drop, film thickness, plug length). The
forward steps and checkpoints run in FP64 (precision=64) or FP32
(precision=32, half the checkpoint memory); the reverse sweep is FP64
(reverse_precision=64, on the stored states widened to FP64) or FP32
(reverse_precision=32, for an FP32 forward: per-step arithmetic in FP32, sums
over steps and nodes in FP64).
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import (LBM_COLL_MRT, LBM_EOS_CS, LBM_EOS_PR, LBM_OK, LBMError, _check, lbm_airway_rho0,
               lbm_airway_rho0_tangent, lbm_collision, lbm_drive, lbm_eos, lbm_grid, lib)

_P = C.c_void_p


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (host or device)."""
    if hasattr(a, "data_ptr"):
        return _P(a.data_ptr())
    return _P(a.ctypes.data)


class Adjoint:
    """Forward run with checkpoints and its adjoint for one channel geometry.

    ``forward(rho0, dp, gx, gy)`` returns (J_tau, J_p); ``backward(w_tau,
    w_p)`` returns the gradient of w_tau J_tau + w_p J_p with respect to rho0
    (array of the input's kind and device) and a dict with dp, gx, gy.
    """

    def __init__(self, nx, ny, nsteps, *, walls=True, bc_x=True, a=1.0, b=4.0, R=1.0, T_over_Tc=0.85,
                 k=1.0, kappa=0.5, tau=1.0, wetting=0.0, p_ref=None, eos="cs", omega=0.344, collision="bgk",
                 s_e=1.64, s_eps=1.54, s_j=1.0, s_q=1.7, s_nu=None, block_steps=0, precision=64, reverse_precision=64, stream=None):
        self.nx, self.ny, self.nsteps = nx, ny, nsteps
        self.grid = lbm_grid(nx, ny, int(walls), int(bc_x), int(precision))
        self.eos = lbm_eos(a, b, R, T_over_Tc, k, kappa, {"cs": LBM_EOS_CS, "pr": LBM_EOS_PR}[eos], omega)
        self.p_ref = math.nan if p_ref is None else p_ref
        self._stream = stream
        h = _P()
        _check(lib().lbm_adjoint_init(C.byref(self.grid), C.byref(self.eos), float(tau), float(wetting),
                                      int(nsteps), int(block_steps),
                                      _P(stream.cuda_stream) if stream is not None else None, C.byref(h)))
        self.h = h
        if collision != "bgk":
            if collision != "mrt":
                raise ValueError(collision)
            coll = lbm_collision(LBM_COLL_MRT, s_e, s_eps, s_j, s_q, 0.0 if s_nu is None else s_nu)
            self._chk(lib().lbm_adjoint_set_collision(self.h, C.byref(coll)))
        if reverse_precision != 64:
            self._chk(lib().lbm_adjoint_set_precision(self.h, int(reverse_precision)))
        self.generation = 0      # forward runs so far (guards stale backward calls)
        self._rho0_like = None

    def _chk(self, st):
        if st != LBM_OK:
            raise LBMError(st, lib().lbm_adjoint_last_error(self.h).decode())

    def forward(self, rho0, dp=0.0, gx=0.0, gy=0.0):
        if hasattr(rho0, "contiguous"):
            import torch
            rho0 = rho0.detach().to(torch.float64).contiguous()
        else:
            rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
        assert tuple(rho0.shape) == (self.ny, self.nx)
        drive = lbm_drive(float(dp), self.p_ref, float(gx), float(gy))
        J = (C.c_double * 2)()
        self._chk(lib().lbm_adjoint_forward(self.h, C.byref(drive), _ptr(rho0), J))
        self._rho0_like = rho0
        self.generation += 1
        return J[0], J[1]

    def backward(self, w_tau=1.0, w_p=0.0):
        like = self._rho0_like
        if like is None:
            raise LBMError(6, "backward before forward")
        if hasattr(like, "data_ptr"):
            import torch
            g = torch.empty_like(like)
        else:
            g = np.empty_like(like)
        gd = (C.c_double * 3)()
        self._chk(lib().lbm_adjoint_backward(self.h, float(w_tau), float(w_p), _ptr(g), gd))
        return g, {"dp": gd[0], "gx": gd[1], "gy": gd[2]}

    def close(self):
        if getattr(self, "h", None):
            lib().lbm_adjoint_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _torch():
    import torch
    return torch


class WallLoads:
    """``WallLoads.apply(adj, rho0, dp, gx, gy) -> (J_tau, J_p)`` (torch scalars)."""

    _fn = None

    @classmethod
    def apply(cls, adj, rho0, dp, gx=None, gy=None):
        if cls._fn is None:
            cls._fn = _make_wall_loads()
        torch = _torch()
        z = torch.zeros((), dtype=torch.float64)
        return cls._fn.apply(adj, rho0, dp, z if gx is None else gx, z if gy is None else gy)


def _make_wall_loads():
    torch = _torch()

    class _WallLoads(torch.autograd.Function):
        @staticmethod
        def forward(ctx, adj, rho0, dp, gx, gy):
            jt, jp = adj.forward(rho0, float(dp), float(gx), float(gy))
            ctx.adj, ctx.gen = adj, adj.generation
            ctx.meta = (rho0.device, dp.device, gx.device, gy.device)
            return (torch.tensor(jt, dtype=torch.float64, device=rho0.device),
                    torch.tensor(jp, dtype=torch.float64, device=rho0.device))

        @staticmethod
        def backward(ctx, g_tau, g_p):
            adj = ctx.adj
            if adj.generation != ctx.gen:
                raise RuntimeError("the adjoint's checkpoints belong to a later forward run")
            w_tau = 0.0 if g_tau is None else float(g_tau)
            w_p = 0.0 if g_p is None else float(g_p)
            g, gd = adj.backward(w_tau, w_p)
            dev_r, dev_dp, dev_gx, dev_gy = ctx.meta
            g = g if hasattr(g, "data_ptr") else torch.from_numpy(g)
            return (None, g.to(dev_r), torch.tensor(gd["dp"], dtype=torch.float64, device=dev_dp),
                    torch.tensor(gd["gx"], dtype=torch.float64, device=dev_gx),
                    torch.tensor(gd["gy"], dtype=torch.float64, device=dev_gy))

    return _WallLoads


class AirwayProfile:
    """``AirwayProfile.apply(film, plug_len, nx, ny, plug_x, rho_l, rho_g, width=4, noise=0, seed=1,
    device='cpu') -> rho0`` (float64 tensor, ny x nx), differentiable in film and plug_len."""

    _fn = None

    @classmethod
    def apply(cls, film, plug_len, nx, ny, plug_x, rho_l, rho_g, width=4.0, noise=0.0, seed=1, device="cpu"):
        if cls._fn is None:
            cls._fn = _make_airway_profile()
        return cls._fn.apply(film, plug_len, (nx, ny, plug_x, rho_l, rho_g, width, noise, seed, device))


def _make_airway_profile():
    torch = _torch()

    class _AirwayProfile(torch.autograd.Function):
        @staticmethod
        def forward(ctx, film, plug_len, consts):
            nx, ny, plug_x, rho_l, rho_g, width, noise, seed, device = consts
            h, L = float(film), float(plug_len)
            rho0 = lbm_airway_rho0(nx, ny, h, plug_x, L, rho_l, rho_g, width, noise, seed)
            d_film, d_plug = lbm_airway_rho0_tangent(nx, ny, h, plug_x, L, rho_l, rho_g, width)
            ctx.save_for_backward(torch.from_numpy(d_film).to(device), torch.from_numpy(d_plug).to(device))
            ctx.devs = (film.device, plug_len.device)
            return torch.from_numpy(rho0).to(device)

        @staticmethod
        def backward(ctx, g):
            d_film, d_plug = ctx.saved_tensors
            return ((g * d_film).sum().to(ctx.devs[0]), (g * d_plug).sum().to(ctx.devs[1]), None)

    return _AirwayProfile

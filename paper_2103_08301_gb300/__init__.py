"""GB300-native EOS-based multiphase lattice Boltzmann solver (arXiv 2103.08301).

A thin ctypes binding of the C ABI declared in ``include/lbm.h``: the same entry
points under the same names, plus a small ``Lattice`` convenience class. The
binding only marshals arguments; every step of the method runs in the CUDA
kernels of ``liblbm.so``. PyTorch is used for device buffers and streams.

The library is built in-tree by ``paper_2103_08301_gb300.build.build()``. If
it is missing this package raises on use: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_OK, LBM_ERR_ARG, LBM_ERR_PARAM, LBM_ERR_CUDA, LBM_ERR_OOM, LBM_ERR_NAN, LBM_ERR_STATE, LBM_ERR_TIMEOUT = range(8)
LBM_OPT_CTAS_PER_SM, LBM_OPT_REVERSE, LBM_OPT_STRIP, LBM_OPT_STAGED, LBM_OPT_GRAPH_STEPS, LBM_OPT_ROWS2, LBM_OPT_TMA = \
    1, 2, 3, 4, 5, 6, 7
LBM_OPT_PREFETCH, LBM_OPT_GENERAL, LBM_OPT_FAULT_SKIP_COPY, LBM_OPT_PERSISTENT, LBM_OPT_BAND, LBM_OPT_PDL, \
    LBM_OPT_TILE = 8, 9, 10, 11, 12, 13, 14


class lbm_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("walls", C.c_int32), ("bc_x", C.c_int32),
                ("precision", C.c_int32)]


class lbm_eos(C.Structure):
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("T_over_Tc", C.c_double),
                ("k", C.c_double), ("kappa", C.c_double), ("kind", C.c_int32), ("omega", C.c_double)]


LBM_EOS_CS, LBM_EOS_PR = 0, 1
LBM_COLL_BGK, LBM_COLL_MRT = 0, 1


class lbm_collision(C.Structure):
    _fields_ = [("kind", C.c_int32), ("s_e", C.c_double), ("s_eps", C.c_double), ("s_j", C.c_double),
                ("s_q", C.c_double), ("s_nu", C.c_double)]


class lbm_drive(C.Structure):
    _fields_ = [("dp", C.c_double), ("p_ref", C.c_double), ("gx", C.c_double), ("gy", C.c_double)]


class lbm_diag_t(C.Structure):
    _fields_ = [("step", C.c_int64), ("mass", C.c_double), ("wall_shear_sum", C.c_double),
                ("tau_wall_min", C.c_double), ("tau_wall_max", C.c_double),
                ("p_wall_min", C.c_double), ("p_wall_max", C.c_double),
                ("nan_detected", C.c_int32), ("pad_", C.c_int32),
                ("T", C.c_double), ("Tc", C.c_double), ("rho_g", C.c_double), ("rho_l", C.c_double),
                ("p_sat", C.c_double), ("rho_in", C.c_double), ("rho_out", C.c_double),
                ("rho_in_l", C.c_double), ("rho_out_l", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


# Every symbol declared in include/lbm.h, with (restype, argtypes).
_P = C.c_void_p
_SIGS = {
    "lbm_workspace_bytes": (C.c_size_t, [C.POINTER(lbm_grid)]),
    "lbm_init": (C.c_int, [C.POINTER(lbm_grid), C.POINTER(lbm_eos), C.c_double, _P, C.c_double,
                           C.POINTER(lbm_drive), C.POINTER(C.c_double), _P, C.c_size_t, _P,
                           C.POINTER(_P)]),
    "lbm_workspace_bytes_inplace": (C.c_size_t, [C.POINTER(lbm_grid)]),
    "lbm_init_inplace": (C.c_int, [C.POINTER(lbm_grid), C.POINTER(lbm_eos), C.c_double, C.c_double,
                                   C.POINTER(lbm_drive), C.POINTER(C.c_double), _P, C.c_size_t, _P,
                                   C.POINTER(_P)]),
    "lbm_step": (C.c_int, [_P, C.c_int64]),
    "lbm_fields": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "lbm_diag": (C.c_int, [_P, C.POINTER(lbm_diag_t)]),
    "lbm_diag_async": (C.c_int, [_P, _P]),
    "lbm_populations": (C.c_int, [_P, _P]),
    "lbm_reset_diag": (C.c_int, [_P]),
    "lbm_batch_reset_diag": (C.c_int, [_P]),
    "lbm_load_populations": (C.c_int, [_P, _P]),
    "lbm_checkpoint_bytes": (C.c_size_t, [_P]),
    "lbm_checkpoint": (C.c_int, [_P, _P, C.c_size_t]),
    "lbm_restore": (C.c_int, [_P, _P, C.c_size_t]),
    "lbm_set_option": (C.c_int, [_P, C.c_int, C.c_int64]),
    "lbm_set_collision": (C.c_int, [_P, C.POINTER(lbm_collision)]),
    "lbm_launch_info": (C.c_int, [_P] + [C.POINTER(C.c_int64)] * 4),
    "lbm_step_noalloc": (C.c_int, [C.POINTER(lbm_grid), C.POINTER(lbm_eos), C.c_double, C.c_double,
                                   C.POINTER(lbm_drive), _P, _P, C.c_int64, _P, _P, _P]),
    "lbm_batch_init": (C.c_int, [C.c_int32, C.POINTER(lbm_grid), C.POINTER(lbm_eos), C.c_double, C.c_double,
                                 C.POINTER(lbm_drive), C.POINTER(C.POINTER(C.c_double)), _P, C.POINTER(_P)]),
    "lbm_batch_step": (C.c_int, [_P, C.c_int64]),
    "lbm_batch_fields": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P]),
    "lbm_batch_diag": (C.c_int, [_P, C.c_int32, C.POINTER(lbm_diag_t)]),
    "lbm_batch_populations": (C.c_int, [_P, C.c_int32, _P]),
    "lbm_batch_set_option": (C.c_int, [_P, C.c_int, C.c_int64]),
    "lbm_batch_set_collision": (C.c_int, [_P, C.POINTER(lbm_collision)]),
    "lbm_batch_launch_info": (C.c_int, [_P] + [C.POINTER(C.c_int64)] * 4),
    "lbm_batch_autotune": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_double)]),
    "lbm_batch_last_error": (C.c_char_p, [_P]),
    "lbm_batch_free": (None, [_P]),
    "lbm_plug_analysis": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_double), C.c_double, _P]),
    "lbm_free": (None, [_P]),
    "lbm_status_string": (C.c_char_p, [C.c_int]),
    "lbm_last_error": (C.c_char_p, [_P]),
    "lbm_coexistence": (C.c_int, [C.POINTER(lbm_eos)] + [C.POINTER(C.c_double)] * 4),
    "lbm_relaxed_coexistence": (C.c_int, [C.POINTER(lbm_eos), C.c_double, C.POINTER(lbm_collision), C.c_int32,
                                          C.c_int32, C.c_int64, _P] + [C.POINTER(C.c_double)] * 4),
    "lbm_airway_rho0": (C.c_int, [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double,
                                  C.c_double, C.c_double, C.c_double, C.c_double, C.c_uint64,
                                  C.POINTER(C.c_double)]),
    "lbm_disk_rho0": (C.c_int, [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double,
                                C.c_double, C.c_double, C.c_double, C.c_double, C.c_uint64,
                                C.POINTER(C.c_double)]),
    "lbm_airway_rho0_tangent": (C.c_int, [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double,
                                          C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double),
                                          C.POINTER(C.c_double)]),
    "lbm_adjoint_init": (C.c_int, [C.POINTER(lbm_grid), C.POINTER(lbm_eos), C.c_double, C.c_double,
                                   C.c_int64, C.c_int64, _P, C.POINTER(_P)]),
    "lbm_adjoint_forward": (C.c_int, [_P, C.POINTER(lbm_drive), _P, C.POINTER(C.c_double)]),
    "lbm_adjoint_backward": (C.c_int, [_P, C.c_double, C.c_double, _P, C.POINTER(C.c_double)]),
    "lbm_adjoint_set_collision": (C.c_int, [_P, C.POINTER(lbm_collision)]),
    "lbm_adjoint_set_precision": (C.c_int, [_P, C.c_int32]),
    "lbm_adjoint_last_error": (C.c_char_p, [_P]),
    "lbm_adjoint_free": (None, [_P]),
}

_lib = None


class LBMError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{status_string(status)} ({status}){': ' + msg if msg else ''}")


def lib():
    """The loaded liblbm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with paper_2103_08301_gb300.build.build() "
                "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(s: int) -> str:
    try:
        return lib().lbm_status_string(int(s)).decode()
    except ImportError:
        return f"status {s}"


def _check(st, ctx=None):
    if st != LBM_OK:
        msg = lib().lbm_last_error(ctx).decode() if ctx else ""
        raise LBMError(st, msg)


# ---------------------------------------------------------------------------
# Functions with the C names (thin wrappers)
# ---------------------------------------------------------------------------

def lbm_workspace_bytes(grid: lbm_grid) -> int:
    return int(lib().lbm_workspace_bytes(C.byref(grid)))


def lbm_init(grid, eos, tau, wetting, drive, rho0, workspace=None, ws_bytes=0, stream=None, wall_mask=None):
    """lbm_init; wall_mask: None or an (ny, nx) array, nonzero = solid node."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    mask = None
    if wall_mask is not None:
        mask = np.ascontiguousarray(np.asarray(wall_mask) != 0, dtype=np.uint8)
        if mask.shape != (grid.ny, grid.nx):
            raise ValueError(f"wall_mask shape {mask.shape} != {(grid.ny, grid.nx)}")
    ctx = _P()
    st = lib().lbm_init(C.byref(grid), C.byref(eos), float(tau),
                        _P(mask.ctypes.data) if mask is not None else None, float(wetting),
                        C.byref(drive) if drive is not None else None,
                        rho0.ctypes.data_as(C.POINTER(C.c_double)),
                        _P(workspace) if workspace else None, int(ws_bytes),
                        _P(stream) if stream else None, C.byref(ctx))
    _check(st)
    return ctx


def lbm_workspace_bytes_inplace(grid: lbm_grid) -> int:
    return int(lib().lbm_workspace_bytes_inplace(C.byref(grid)))


def lbm_init_inplace(grid, eos, tau, wetting, drive, rho0, workspace=None, ws_bytes=0, stream=None):
    """lbm_init_inplace: a context with one population array (in-place streaming)."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    ctx = _P()
    st = lib().lbm_init_inplace(C.byref(grid), C.byref(eos), float(tau), float(wetting),
                                C.byref(drive) if drive is not None else None,
                                rho0.ctypes.data_as(C.POINTER(C.c_double)),
                                _P(workspace) if workspace else None, int(ws_bytes),
                                _P(stream) if stream else None, C.byref(ctx))
    _check(st)
    return ctx


def lbm_step(ctx, n: int) -> int:
    return int(lib().lbm_step(ctx, int(n)))


def lbm_step_noalloc(grid, eos, tau, wetting, drive, f_in_ptr, f_out_ptr, ctas=0, diag_ptr=None,
                     stream=None, err_ptr=None) -> int:
    """One step between caller-owned device buffers (raw pointers); returns the status."""
    return int(lib().lbm_step_noalloc(C.byref(grid), C.byref(eos), float(tau), float(wetting),
                                      C.byref(drive) if drive is not None else None,
                                      _P(f_in_ptr), _P(f_out_ptr), int(ctas),
                                      _P(diag_ptr) if diag_ptr else None, _P(err_ptr) if err_ptr else None,
                                      _P(stream) if stream else None))


class lbm_plug_state(C.Structure):
    _fields_ = [("x_rear", C.c_double), ("x_front", C.c_double), ("intact", C.c_int32),
                ("n_droplets", C.c_int32), ("droplet_mass", C.c_double), ("wall_liquid_mass", C.c_double)]


def lbm_plug_analysis(rho, rho_mid):
    """Plug interfaces, rupture state and aerosol droplets of a channel density field."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ny, nx = rho.shape
    st = lbm_plug_state()
    _check(lib().lbm_plug_analysis(nx, ny, rho.ctypes.data_as(C.POINTER(C.c_double)), float(rho_mid),
                                   _P(C.addressof(st))))
    return {k: getattr(st, k) for k, _ in st._fields_}


def lbm_coexistence(eos: lbm_eos):
    Tc, g, l, p = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    _check(lib().lbm_coexistence(C.byref(eos), C.byref(Tc), C.byref(g), C.byref(l), C.byref(p)))
    return Tc.value, g.value, l.value, p.value


def lbm_relaxed_coexistence(eos: lbm_eos, tau=1.0, collision=None, precision=64, ny=192, steps=40000,
                            stream=None):
    """The method's own coexistence from a relaxed flat slab on the GPU:
    dict(rho_g, rho_l, p_gas, p_liq) (mesh pressures k^2 p0)."""
    v = [C.c_double() for _ in range(4)]
    _check(lib().lbm_relaxed_coexistence(C.byref(eos), float(tau), C.byref(collision) if collision else None,
                                         int(precision), int(ny), int(steps),
                                         _P(stream.cuda_stream) if stream is not None else None,
                                         *[C.byref(x) for x in v]))
    return dict(zip(("rho_g", "rho_l", "p_gas", "p_liq"), [x.value for x in v]))


def lbm_airway_rho0(nx, ny, film, plug_x, plug_len, rho_l, rho_g, width=4.0, noise=0.0, seed=1):
    out = np.empty((ny, nx), dtype=np.float64)
    _check(lib().lbm_airway_rho0(nx, ny, film, plug_x, plug_len, rho_l, rho_g, width, noise, seed,
                                 out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def lbm_airway_rho0_tangent(nx, ny, film, plug_x, plug_len, rho_l, rho_g, width=4.0):
    """(d rho0 / d film, d rho0 / d plug_len) of the noise-free airway profile."""
    d_film = np.empty((ny, nx), dtype=np.float64)
    d_plug = np.empty((ny, nx), dtype=np.float64)
    _check(lib().lbm_airway_rho0_tangent(nx, ny, film, plug_x, plug_len, rho_l, rho_g, width,
                                         d_film.ctypes.data_as(C.POINTER(C.c_double)),
                                         d_plug.ctypes.data_as(C.POINTER(C.c_double))))
    return d_film, d_plug


def lbm_disk_rho0(nx, ny, cx, cy, r0, rho_l, rho_g, width=4.0, noise=0.0, seed=1):
    out = np.empty((ny, nx), dtype=np.float64)
    _check(lib().lbm_disk_rho0(nx, ny, cx, cy, r0, rho_l, rho_g, width, noise, seed,
                               out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


# ---------------------------------------------------------------------------
# Convenience class
# ---------------------------------------------------------------------------

class Lattice:
    """One channel (or periodic box) resident on the current CUDA device.

    Parameters mirror lbm_init; ``mask`` is the wall mask, an (ny, nx) array
    with nonzero entries at solid nodes. ``workspace`` may be a CUDA torch tensor of at
    least ``lbm_workspace_bytes`` bytes (kept alive by this object); by default
    the library allocates. ``stream`` is a torch.cuda.Stream or None.
    ``inplace=True`` builds the context with lbm_init_inplace (one population
    array, in-place streaming; no mask; workspace of lbm_workspace_bytes_inplace).
    """

    def __init__(self, nx, ny, rho0, *, walls=False, bc_x=False, precision=32, a=1.0, b=4.0,
                 R=1.0, T_over_Tc=0.8, k=1.0, kappa=0.5, tau=1.0, wetting=0.0, dp=0.0,
                 p_ref=None, gx=0.0, gy=0.0, eos="cs", omega=0.344, collision="bgk", s_e=1.64,
                 s_eps=1.54, s_j=1.0, s_q=1.7, s_nu=None, workspace=None, stream=None, mask=None,
                 inplace=False):
        self.grid = lbm_grid(nx, ny, int(walls), int(bc_x), int(precision))
        self.eos = lbm_eos(a, b, R, T_over_Tc, k, kappa, {"cs": LBM_EOS_CS, "pr": LBM_EOS_PR}[eos], omega)
        self.drive = lbm_drive(dp, math.nan if p_ref is None else p_ref, gx, gy)
        self.nx, self.ny, self.precision = nx, ny, precision
        self.dtype = np.float32 if precision == 32 else np.float64
        self._ws = workspace
        self._stream = stream
        ws_ptr, ws_bytes = None, 0
        if workspace is not None:
            ws_ptr, ws_bytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
        sptr = stream.cuda_stream if stream is not None else None
        if inplace:
            if mask is not None:
                raise ValueError("in-place contexts take no wall mask")
            self.ctx = lbm_init_inplace(self.grid, self.eos, tau, wetting, self.drive, rho0, ws_ptr, ws_bytes, sptr)
        else:
            self.ctx = lbm_init(self.grid, self.eos, tau, wetting, self.drive, rho0, ws_ptr, ws_bytes, sptr,
                                wall_mask=mask)
        if collision != "bgk":
            if collision != "mrt":
                raise ValueError(collision)
            self.set_collision(lbm_collision(LBM_COLL_MRT, s_e, s_eps, s_j, s_q, 0.0 if s_nu is None else s_nu))

    def set_collision(self, coll):
        """lbm_set_collision with an lbm_collision (None: BGK)."""
        _check(lib().lbm_set_collision(self.ctx, C.byref(coll) if coll is not None else None), self.ctx)

    # -- stepping -----------------------------------------------------------
    def step(self, n=1):
        st = lbm_step(self.ctx, n)
        if st == LBM_ERR_NAN:
            raise LBMError(st, "a step met a non-finite or non-positive density")
        _check(st, self.ctx)

    # -- outputs ------------------------------------------------------------
    def fields(self):
        """dict(rho, vx, vy, tau_wall[2, nx], p_wall[2, nx]) as numpy arrays."""
        ny, nx, dt = self.ny, self.nx, self.dtype
        out = {k: np.zeros((ny, nx), dt) for k in ("rho", "vx", "vy")}
        out["tau_wall"] = np.zeros((2, nx), dt)
        out["p_wall"] = np.zeros((2, nx), dt)
        p = [_P(out[k].ctypes.data) for k in ("rho", "vx", "vy", "tau_wall", "p_wall")]
        _check(lib().lbm_fields(self.ctx, *p), self.ctx)
        return out

    def fields_into(self, rho=None, vx=None, vy=None, tau_wall=None, p_wall=None):
        """Write fields into caller buffers (CUDA torch tensors or numpy arrays)."""
        def ptr(t):
            if t is None:
                return None
            return _P(t.data_ptr()) if hasattr(t, "data_ptr") else _P(t.ctypes.data)
        _check(lib().lbm_fields(self.ctx, ptr(rho), ptr(vx), ptr(vy), ptr(tau_wall), ptr(p_wall)), self.ctx)

    def diag(self):
        d = lbm_diag_t()
        _check(lib().lbm_diag(self.ctx, C.byref(d)), self.ctx)
        return d.as_dict()

    def diag_async(self, dst):
        """lbm_diag_async into `dst` (7 float64: a pinned host or device torch
        tensor, or a numpy array in pinned memory); valid once the stream has
        passed this point."""
        ptr = dst.data_ptr() if hasattr(dst, "data_ptr") else dst.ctypes.data
        _check(lib().lbm_diag_async(self.ctx, _P(ptr)), self.ctx)

    def reset_diag(self):
        """lbm_reset_diag: the accumulators restart from the next step."""
        _check(lib().lbm_reset_diag(self.ctx), self.ctx)

    def populations(self):
        f = np.empty((9, self.ny, self.nx), self.dtype)
        _check(lib().lbm_populations(self.ctx, _P(f.ctypes.data)), self.ctx)
        return f

    def load_populations(self, f):
        f = np.ascontiguousarray(f, dtype=self.dtype)
        assert f.shape == (9, self.ny, self.nx)
        _check(lib().lbm_load_populations(self.ctx, _P(f.ctypes.data)), self.ctx)

    def checkpoint(self):
        n = int(lib().lbm_checkpoint_bytes(self.ctx))
        buf = np.empty(n, np.uint8)
        _check(lib().lbm_checkpoint(self.ctx, _P(buf.ctypes.data), n), self.ctx)
        return buf

    def restore(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib().lbm_restore(self.ctx, _P(buf.ctypes.data), buf.size), self.ctx)

    def set_option(self, opt, value):
        _check(lib().lbm_set_option(self.ctx, int(opt), int(value)), self.ctx)

    def launch_info(self):
        a, b, c, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        _check(lib().lbm_launch_info(self.ctx, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), self.ctx)
        return {"ctas": a.value, "threads": b.value, "units": c.value, "staged": bool(d.value)}

    def close(self):
        if getattr(self, "ctx", None):
            lib().lbm_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many channels of different sizes and drives stepped together.

    channels: list of dicts with nx, ny, rho0 (ny x nx array) and optionally
    dp, p_ref, gx, gy. Shared keyword arguments as for Lattice.
    """

    def __init__(self, channels, *, walls=True, bc_x=True, precision=32, a=1.0, b=4.0, R=1.0,
                 T_over_Tc=0.85, k=1.0, kappa=0.5, tau=1.0, wetting=0.0, stream=None):
        n = len(channels)
        self.n = n
        self.precision = precision
        self.dtype = np.float32 if precision == 32 else np.float64
        self.shapes = [(c["ny"], c["nx"]) for c in channels]
        grids = (lbm_grid * n)(*[lbm_grid(c["nx"], c["ny"], int(walls), int(bc_x), int(precision))
                                 for c in channels])
        drives = (lbm_drive * n)(*[lbm_drive(c.get("dp", 0.0), math.nan if c.get("p_ref") is None else c["p_ref"],
                                             c.get("gx", 0.0), c.get("gy", 0.0)) for c in channels])
        self._rho0 = [np.ascontiguousarray(c["rho0"], dtype=np.float64) for c in channels]
        ptrs = (C.POINTER(C.c_double) * n)(*[r.ctypes.data_as(C.POINTER(C.c_double)) for r in self._rho0])
        self.eos = lbm_eos(a, b, R, T_over_Tc, k, kappa)
        self._stream = stream
        h = _P()
        _check(lib().lbm_batch_init(n, grids, C.byref(self.eos), float(tau), float(wetting), drives, ptrs,
                                    _P(stream.cuda_stream) if stream is not None else None, C.byref(h)))
        self.h = h

    def _chk(self, st):
        if st != LBM_OK:
            raise LBMError(st, lib().lbm_batch_last_error(self.h).decode())

    def step(self, n=1):
        st = lib().lbm_batch_step(self.h, int(n))
        if st == LBM_ERR_NAN:
            raise LBMError(st, "a step met a non-finite or non-positive density")
        self._chk(st)

    def fields(self, c):
        ny, nx = self.shapes[c]
        out = {k: np.zeros((ny, nx), self.dtype) for k in ("rho", "vx", "vy")}
        out["tau_wall"] = np.zeros((2, nx), self.dtype)
        out["p_wall"] = np.zeros((2, nx), self.dtype)
        p = [_P(out[k].ctypes.data) for k in ("rho", "vx", "vy", "tau_wall", "p_wall")]
        self._chk(lib().lbm_batch_fields(self.h, int(c), *p))
        return out

    def diag(self, c):
        d = lbm_diag_t()
        self._chk(lib().lbm_batch_diag(self.h, int(c), C.byref(d)))
        return d.as_dict()

    def populations(self, c):
        ny, nx = self.shapes[c]
        f = np.empty((9, ny, nx), self.dtype)
        self._chk(lib().lbm_batch_populations(self.h, int(c), _P(f.ctypes.data)))
        return f

    def set_option(self, opt, value):
        self._chk(lib().lbm_batch_set_option(self.h, int(opt), int(value)))

    def reset_diag(self):
        self._chk(lib().lbm_batch_reset_diag(self.h))

    def set_collision(self, coll):
        """lbm_batch_set_collision with an lbm_collision (None: BGK)."""
        self._chk(lib().lbm_batch_set_collision(self.h, C.byref(coll) if coll is not None else None))

    def launch_info(self):
        v = [C.c_int64() for _ in range(4)]
        self._chk(lib().lbm_batch_launch_info(self.h, *[C.byref(x) for x in v]))
        return dict(zip(("ctas", "segments", "staged", "strip"), [x.value for x in v]))

    def autotune(self, trial_steps=20):
        c, w, ms = C.c_int64(), C.c_int64(), C.c_double()
        self._chk(lib().lbm_batch_autotune(self.h, int(trial_steps), C.byref(c), C.byref(w), C.byref(ms)))
        return {"ctas_per_sm": c.value, "strip": w.value, "ms_per_step": ms.value}

    def close(self):
        if getattr(self, "h", None):
            lib().lbm_batch_free(self.h)
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

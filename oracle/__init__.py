"""FP64 CPU oracle of the EOS-based multiphase LBM step (arXiv 2103.08301).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package. The CUDA
product path (``paper_2103_08301_gb300``) does not import it, shares no code
with it, and must keep working when this directory is absent.

The arithmetic lives in ``lbm_oracle.c`` (plain C, double precision, one pass
per algorithmic step). This module compiles it with gcc and exposes it to
numpy through ctypes. Every function cites the part of the paper it follows
in the C source.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(closed forms, library routines, physics laws); none is "parity unpinned".
The boundary arithmetic (pressure-column branch roots, spinodal saturation,
the column density blend and extrapolation, the kappa terms of the wall
pressure, the wetting offset) is pinned in ``tests/test_oracle_boundaries.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
Q = 9


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (portable flags, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("walls", C.c_int32), ("bc_x", C.c_int32),
                ("a", C.c_double), ("b", C.c_double), ("R", C.c_double), ("T", C.c_double),
                ("k", C.c_double), ("kappa", C.c_double), ("tau", C.c_double), ("wet", C.c_double),
                ("rho_in_g", C.c_double), ("rho_in_l", C.c_double), ("rho_out_g", C.c_double),
                ("rho_out_l", C.c_double), ("ph_g", C.c_double), ("ph_l", C.c_double),
                ("gx", C.c_double), ("gy", C.c_double),
                ("eos_kind", C.c_int32), ("collision", C.c_int32), ("aalpha", C.c_double),
                ("s_e", C.c_double), ("s_eps", C.c_double), ("s_j", C.c_double), ("s_q", C.c_double),
                ("s_nu", C.c_double), ("mask", C.c_void_p)]


class Eos(C.Structure):
    _fields_ = [("kind", C.c_int32), ("a", C.c_double), ("b", C.c_double), ("R", C.c_double),
                ("T", C.c_double), ("aalpha", C.c_double)]


class Diag(C.Structure):
    _fields_ = [("mass", C.c_double), ("J", C.c_double), ("tw_min", C.c_double),
                ("tw_max", C.c_double), ("pw_min", C.c_double), ("pw_max", C.c_double),
                ("Jp", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_D = C.c_double
_PD = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        for name in ("orc_cs_p0", "orc_cs_dp0", "orc_cs_mu"):
            getattr(L, name).restype = _D
            getattr(L, name).argtypes = [_D] * 5
        L.orc_cs_critical.argtypes = [_D, _D, _D, _PD, _PD]
        L.orc_maxwell.argtypes = [_D, _D, _D, _D, _PD, _PD, _PD]
        L.orc_gas_root.argtypes = [_D, _D, _D, _D, _D, _PD]
        L.orc_liquid_root.argtypes = [_D, _D, _D, _D, _D, _PD]
        for name in ("orc_eos_p0", "orc_eos_dp0", "orc_eos_mu"):
            getattr(L, name).restype = _D
            getattr(L, name).argtypes = [C.POINTER(Eos), _D]
        L.orc_pr_alpha.restype = _D
        L.orc_pr_alpha.argtypes = [_D, _D]
        L.orc_eos_critical.argtypes = [C.c_int, _D, _D, _D, _PD, _PD]
        L.orc_eos_maxwell.argtypes = [C.POINTER(Eos), _PD, _PD, _PD]
        L.orc_eos_gas_root.argtypes = [C.POINTER(Eos), _D, _PD]
        L.orc_eos_liquid_root.argtypes = [C.POINTER(Eos), _D, _PD]
        L.orc_eos_column_density.argtypes = [C.POINTER(Eos), C.c_int, _D, _PD, C.POINTER(C.c_int)]
        L.orc_mrt_moments.argtypes = [_PD, _PD]
        L.orc_mrt_moments.restype = None
        L.orc_feq.argtypes = [_D, _D, _D, _PD]
        L.orc_feq.restype = None
        L.orc_grad_periodic.argtypes = [C.c_int, C.c_int, _PD, _PD, _PD]
        L.orc_grad_periodic.restype = None
        L.orc_lap_periodic.argtypes = [C.c_int, C.c_int, _PD, _PD]
        L.orc_lap_periodic.restype = None
        L.orc_init.argtypes = [C.POINTER(Params), _PD, _PD]
        L.orc_init.restype = None
        L.orc_step.argtypes = [C.POINTER(Params), _PD, _PD, C.POINTER(Diag)]
        L.orc_run.argtypes = [C.POINTER(Params), _PD, C.c_long, C.POINTER(Diag)]
        L.orc_fields.argtypes = [C.POINTER(Params), _PD, _PD, _PD, _PD, _PD, _PD]
        L.orc_force.argtypes = [C.POINTER(Params), _PD, _PD, _PD]
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
        L.orc_set_num_threads.restype = None
        _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_PD)


# --------------------------------------------------------------------------
# Equation of state (Carnahan-Starling)
# --------------------------------------------------------------------------

def cs_p0(a, b, R, T, rho):
    return lib().orc_cs_p0(a, b, R, T, rho)


def cs_dp0(a, b, R, T, rho):
    return lib().orc_cs_dp0(a, b, R, T, rho)


def cs_mu(a, b, R, T, rho):
    return lib().orc_cs_mu(a, b, R, T, rho)


def cs_critical(a=1.0, b=4.0, R=1.0):
    Tc, rc = _D(), _D()
    if lib().orc_cs_critical(a, b, R, C.byref(Tc), C.byref(rc)):
        raise ValueError("bad EOS parameters")
    return Tc.value, rc.value


def maxwell(a, b, R, T):
    """(rho_g, rho_l, p_sat) of the Maxwell construction at absolute T."""
    g, l, p = _D(), _D(), _D()
    if lib().orc_maxwell(a, b, R, T, C.byref(g), C.byref(l), C.byref(p)):
        raise ValueError("no coexistence (T >= Tc)")
    return g.value, l.value, p.value


def gas_root(a, b, R, T, p0_target):
    r = _D()
    if lib().orc_gas_root(a, b, R, T, p0_target, C.byref(r)):
        raise ValueError("pressure outside the gas branch")
    return r.value


def liquid_root(a, b, R, T, p0_target):
    r = _D()
    if lib().orc_liquid_root(a, b, R, T, p0_target, C.byref(r)):
        raise ValueError("pressure outside the liquid branch")
    return r.value


# --------------------------------------------------------------------------
# Equation of state, either kind (0 Carnahan-Starling, 1 Peng-Robinson)
# --------------------------------------------------------------------------

EOS_KINDS = {"cs": 0, "pr": 1}


def pr_alpha(omega, T_over_Tc):
    return lib().orc_pr_alpha(omega, T_over_Tc)


def eos_critical(kind="cs", a=1.0, b=4.0, R=1.0):
    Tc, rc = _D(), _D()
    if lib().orc_eos_critical(EOS_KINDS[kind], a, b, R, C.byref(Tc), C.byref(rc)):
        raise ValueError("bad EOS parameters")
    return Tc.value, rc.value


def eos_p0(e: Eos, rho):
    return lib().orc_eos_p0(C.byref(e), rho)


def eos_dp0(e: Eos, rho):
    return lib().orc_eos_dp0(C.byref(e), rho)


def eos_mu(e: Eos, rho):
    return lib().orc_eos_mu(C.byref(e), rho)


def eos_maxwell(e: Eos):
    g, l, p = _D(), _D(), _D()
    if lib().orc_eos_maxwell(C.byref(e), C.byref(g), C.byref(l), C.byref(p)):
        raise ValueError("no coexistence (T >= Tc)")
    return g.value, l.value, p.value


def eos_gas_root(e: Eos, p0_target):
    r = _D()
    if lib().orc_eos_gas_root(C.byref(e), p0_target, C.byref(r)):
        raise ValueError("pressure outside the gas branch")
    return r.value


def eos_liquid_root(e: Eos, p0_target):
    r = _D()
    if lib().orc_eos_liquid_root(C.byref(e), p0_target, C.byref(r)):
        raise ValueError("pressure outside the liquid branch")
    return r.value


def eos_column_density(e: Eos, liquid: bool, p0_target):
    """(density, saturated) of a pressure column on one branch; a pressure beyond
    the branch's end gives its spinodal density."""
    r, sat = _D(), C.c_int()
    if lib().orc_eos_column_density(C.byref(e), int(liquid), p0_target, C.byref(r), C.byref(sat)):
        raise ValueError("no column density on this branch")
    return r.value, bool(sat.value)


def mrt_moments(f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    m = np.zeros(Q)
    lib().orc_mrt_moments(_ptr(f), _ptr(m))
    return m


def feq(rho, ux, uy):
    out = np.zeros(Q)
    lib().orc_feq(rho, ux, uy, _ptr(out))
    return out


def grad_periodic(psi: np.ndarray):
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    ny, nx = psi.shape
    gx, gy = np.zeros_like(psi), np.zeros_like(psi)
    lib().orc_grad_periodic(nx, ny, _ptr(psi), _ptr(gx), _ptr(gy))
    return gx, gy


def lap_periodic(psi: np.ndarray):
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    ny, nx = psi.shape
    out = np.zeros_like(psi)
    lib().orc_lap_periodic(nx, ny, _ptr(psi), _ptr(out))
    return out


# --------------------------------------------------------------------------
# Simulation
# --------------------------------------------------------------------------

@dataclass
class Setup:
    """Physical set-up of one channel or periodic box (mesh units)."""
    nx: int
    ny: int
    walls: bool = False
    bc_x: bool = False          # pressure inlet / outlet columns
    a: float = 1.0
    b: float = 4.0
    R: float = 1.0
    T_over_Tc: float = 0.8
    k: float = 1.0
    kappa: float = 1.0
    tau: float = 1.0
    wet: float = 0.0
    dp: float = 0.0             # pressure drop between inlet and outlet (mesh units)
    p_ref: float | None = None  # None: k^2 p_sat(T)
    gx: float = 0.0
    gy: float = 0.0
    eos: str = "cs"             # "cs" Carnahan-Starling, "pr" Peng-Robinson (Eq. 2.18)
    omega: float = 0.344        # PR acentric factor (water)
    collision: str = "bgk"      # "bgk" or "mrt" (Eq. 2.1)
    s_e: float = 1.64           # MRT rates (Sec. 2.1); s_nu None -> 1/tau
    s_eps: float = 1.54
    s_q: float = 1.7
    s_j: float = 1.0
    s_nu: float | None = None
    mask: np.ndarray | None = None  # (ny, nx), nonzero = solid node (general wall geometry)
    T: float = field(init=False)
    aalpha: float = field(init=False, default=0.0)
    rho_in: float = field(init=False, default=0.0)    # gas-branch column densities
    rho_out: float = field(init=False, default=0.0)
    rho_in_l: float = field(init=False, default=0.0)  # liquid-branch column densities
    rho_out_l: float = field(init=False, default=0.0)
    ph_g: float = field(init=False, default=0.0)      # phase-indicator end points
    ph_l: float = field(init=False, default=0.0)

    def eos_spec(self) -> Eos:
        return Eos(EOS_KINDS[self.eos], self.a, self.b, self.R, self.T, self.aalpha)

    def __post_init__(self):
        if self.mask is not None:
            self.mask = np.ascontiguousarray(np.asarray(self.mask) != 0, dtype=np.uint8)
            assert self.mask.shape == (self.ny, self.nx)
        Tc, _ = eos_critical(self.eos, self.a, self.b, self.R)
        self.T = self.T_over_Tc * Tc
        if self.eos == "pr":
            self.aalpha = self.a * pr_alpha(self.omega, self.T_over_Tc)
        e = self.eos_spec()
        if self.bc_x:
            k2 = self.k * self.k
            below = self.T < Tc
            if self.p_ref is None:
                _, _, psat = eos_maxwell(e)
                pref = k2 * psat
            else:
                pref = self.p_ref
            pin, pout = (pref + 0.5 * self.dp) / k2, (pref - 0.5 * self.dp) / k2
            self.rho_in, _ = eos_column_density(e, False, pin)
            self.rho_out, _ = eos_column_density(e, False, pout)
            if below:
                self.ph_g, self.ph_l, _ = eos_maxwell(e)
                self.rho_in_l, _ = eos_column_density(e, True, pin)
                self.rho_out_l, _ = eos_column_density(e, True, pout)
            else:
                self.rho_in_l, self.rho_out_l = self.rho_in, self.rho_out

    def coexistence(self):
        return eos_maxwell(self.eos_spec())

    def params(self) -> Params:
        s_nu = 1.0 / self.tau if self.s_nu is None else self.s_nu
        return Params(self.nx, self.ny, int(self.walls), int(self.bc_x), self.a, self.b, self.R,
                      self.T, self.k, self.kappa, self.tau, self.wet, self.rho_in, self.rho_in_l,
                      self.rho_out, self.rho_out_l, self.ph_g, self.ph_l, self.gx, self.gy,
                      EOS_KINDS[self.eos], int(self.collision == "mrt"), self.aalpha,
                      self.s_e, self.s_eps, self.s_j, self.s_q, s_nu,
                      None if self.mask is None else self.mask.ctypes.data)


def init(setup: Setup, rho0: np.ndarray) -> np.ndarray:
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    assert rho0.shape == (setup.ny, setup.nx)
    f = np.zeros((Q, setup.ny, setup.nx))
    p = setup.params()
    lib().orc_init(C.byref(p), _ptr(rho0), _ptr(f))
    return f


def step(setup: Setup, f: np.ndarray):
    """One step; returns (f_next, diagnostics of the state read)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    d = Diag()
    p = setup.params()
    if lib().orc_step(C.byref(p), _ptr(f), _ptr(out), C.byref(d)):
        raise MemoryError("oracle step")
    return out, d.as_dict()


def run(setup: Setup, f: np.ndarray, nsteps: int):
    """nsteps steps; returns (f_final, accumulated diagnostics)."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    d = Diag()
    p = setup.params()
    if lib().orc_run(C.byref(p), _ptr(f), int(nsteps), C.byref(d)):
        raise MemoryError("oracle run")
    return f, d.as_dict()


def fields(setup: Setup, f: np.ndarray):
    """dict(rho, vx, vy, tau_wall[2, nx], p_wall[2, nx]) of state f."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    ny, nx = setup.ny, setup.nx
    rho, vx, vy = (np.zeros((ny, nx)) for _ in range(3))
    tw, pw = np.zeros((2, nx)), np.zeros((2, nx))
    p = setup.params()
    if lib().orc_fields(C.byref(p), _ptr(f), _ptr(rho), _ptr(vx), _ptr(vy), _ptr(tw), _ptr(pw)):
        raise MemoryError("oracle fields")
    return {"rho": rho, "vx": vx, "vy": vy, "tau_wall": tw, "p_wall": pw}


def force(setup: Setup, f: np.ndarray):
    f = np.ascontiguousarray(f, dtype=np.float64)
    Fx = np.zeros((setup.ny, setup.nx))
    Fy = np.zeros_like(Fx)
    p = setup.params()
    if lib().orc_force(C.byref(p), _ptr(f), _ptr(Fx), _ptr(Fy)):
        raise MemoryError("oracle force")
    return Fx, Fy


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (for timing it on one core)."""
    lib().orc_set_num_threads(int(n))

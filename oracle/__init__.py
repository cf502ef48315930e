"""FP64 CPU oracle for the SL-MPP5/7 Vlasov-Poisson method (Tanaka et al. 2017).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may import this package.  The product
(the CUDA library and its binding) never imports it, and it never imports the
product: the two share no code.

The arithmetic lives in ``vp_oracle.c`` (plain C, double precision, one
function per step of the paper).  This module compiles it with gcc on first
use and exposes it through ctypes with numpy arrays.

Functions that have no independent pin say so in their docstring
("parity unpinned"); every other one is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle_vp.so")
_SRC = os.path.join(_HERE, "vp_oracle.c")
_lock = threading.Lock()
_lib = None

BC_PERIODIC, BC_OUTFLOW = 0, 1
POIS_PERIODIC, POIS_ISOLATED = 0, 1
SPLIT_KDK, SPLIT_DKD = 0, 1
IC_LANDAU, IC_TWOSTREAM, IC_PLUMMER, IC_ADVECT, IC_SPHERE = 0, 1, 2, 3, 4
NDIAG = 9
DIAG_NAMES = ("mass", "ke", "fe", "pe", "min_f", "max_f", "mode_amp", "l1", "l2")


def build(force: bool = False) -> str:
    """Compile vp_oracle.c into a shared library (OpenMP if available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(_SRC),
                                             os.path.getmtime(os.path.join(_HERE, "vp_oracle.h")))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


class Grid(ctypes.Structure):
    """Mirror of vpo_grid (oracle's own struct)."""
    _fields_ = [
        ("dx", ctypes.c_int), ("dv", ctypes.c_int),
        ("nx", ctypes.c_int * 3), ("nv", ctypes.c_int * 3),
        ("xlo", ctypes.c_double * 3), ("xhi", ctypes.c_double * 3),
        ("vlo", ctypes.c_double * 3), ("vhi", ctypes.c_double * 3),
        ("xbc", ctypes.c_int), ("order", ctypes.c_int), ("mp", ctypes.c_int),
        ("pp", ctypes.c_int), ("alpha", ctypes.c_double),
        ("poisson", ctypes.c_int), ("pois_order", ctypes.c_int),
        ("coupling", ctypes.c_double), ("rho_bg", ctypes.c_double),
    ]

    @property
    def NX(self) -> int:
        return int(np.prod([self.nx[d] for d in range(self.dx)]))

    @property
    def NV(self) -> int:
        return int(np.prod([self.nv[d] for d in range(self.dv)]))

    @property
    def shape(self) -> tuple:
        return tuple(self.nx[d] for d in range(self.dx)) + tuple(self.nv[d] for d in range(self.dv))

    def x_centres(self, d: int) -> np.ndarray:
        h = (self.xhi[d] - self.xlo[d]) / self.nx[d]
        return self.xlo[d] + (np.arange(self.nx[d]) + 0.5) * h

    def v_centres(self, d: int) -> np.ndarray:
        h = (self.vhi[d] - self.vlo[d]) / self.nv[d]
        return self.vlo[d] + (np.arange(self.nv[d]) + 0.5) * h


def grid(dims: int, nx, nv, xlo, xhi, vlo, vhi, *, xbc: int = BC_PERIODIC, order: int = 7,
         mp: int = 1, pp: int = 1, alpha: float = 4.0, poisson: int = POIS_PERIODIC,
         pois_order: int = 6, coupling: float = -1.0, rho_bg: float = 1.0, **_ignored) -> Grid:
    """Build a Grid from plain values (sequences of length `dims`)."""
    g = Grid()
    g.dx = g.dv = dims
    for d in range(dims):
        g.nx[d], g.nv[d] = int(nx[d]), int(nv[d])
        g.xlo[d], g.xhi[d] = float(xlo[d]), float(xhi[d])
        g.vlo[d], g.vhi[d] = float(vlo[d]), float(vhi[d])
    for d in range(dims, 3):
        g.nx[d] = g.nv[d] = 1
    g.xbc, g.order, g.mp, g.pp, g.alpha = xbc, order, mp, pp, float(alpha)
    g.poisson, g.pois_order = poisson, pois_order
    g.coupling, g.rho_bg = float(coupling), float(rho_bg)
    return g


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D, I, L, P = ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_void_p
        GP = ctypes.POINTER(Grid)
        sig = {
            "vpo_csl_flux": (D, [I, D, P]),
            "vpo_mp_constraint": (D, [D, P, D]),
            "vpo_mp_bounds": (None, [P, D, P, P]),
            "vpo_pp_limiter": (D, [D, D, D, D]),
            "vpo_interface_flux": (D, [I, I, I, D, D, P]),
            "vpo_shift_split": (None, [D, P, P]),
            "vpo_advect_line": (None, [I, I, I, D, I, L, P, L, D]),
            "vpo_nx_total": (L, [GP]),
            "vpo_nv_total": (L, [GP]),
            "vpo_rk_mpp5_line": (I, [I, I, D, I, L, P, L, D]),
            "vpo_drift_sweep_rk": (I, [GP, P, I, D]),
            "vpo_kick_sweep_rk": (I, [GP, P, I, D, P]),
            "vpo_drift_sweep": (I, [GP, P, I, D]),
            "vpo_kick_sweep": (I, [GP, P, I, D, P]),
            "vpo_drift_unsplit": (I, [GP, P, D]),
            "vpo_density_moment": (None, [GP, P, P]),
            "vpo_poisson_solve": (I, [GP, P, P, P]),
            "vpo_diagnostics": (None, [GP, P, P, P, P, I, P]),
            "vpo_step": (I, [GP, P, D, I, I, P, I, P]),
            "vpo_init_f": (I, [GP, I, P, I, P]),
            "vpo_cfl_dt": (D, [GP, D, P]),
            "vpo_dft_lines": (None, [L, L, P, L, P, P, I]),
            "vpo_set_threads": (None, [I]),
            "vpo_get_threads": (I, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    _load().vpo_set_threads(int(n))


def get_threads() -> int:
    return int(_load().vpo_get_threads())


# ---- one interface -------------------------------------------------------

def _stencil(u) -> np.ndarray:
    u = _f64(u)
    if u.shape != (7,):
        raise ValueError("stencil must hold u[-3..3] (7 values)")
    return u


def csl_flux(order: int, nu: float, u) -> float:
    """CSL5/CSL7 flux (Sec. 2.1.2) for the stencil u[-3..3], upwind cell u[0]."""
    u = _stencil(u)
    return _load().vpo_csl_flux(order, nu, ctypes.c_void_p(u.ctypes.data + 3 * 8))


def mp_constraint(phi: float, u, alpha: float = 4.0) -> float:
    """MP constraint of Appendix A; u[-3..3] with u[0] the paper's f_i."""
    u = _stencil(u)
    return _load().vpo_mp_constraint(phi, ctypes.c_void_p(u.ctypes.data + 3 * 8), alpha)


def mp_bounds(u, alpha: float = 4.0) -> tuple:
    """(f_min, f_max) of Appendix A steps 4-6 for the stencil u[-3..3], u[0] = f_i."""
    u = _stencil(u)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _load().vpo_mp_bounds(ctypes.c_void_p(u.ctypes.data + 3 * 8), alpha, ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def pp_limiter(phibar: float, u0: float, u1: float, nu: float) -> float:
    """PP flux limiter of Sec. 2.1.1 (Eqs. 15-23)."""
    return _load().vpo_pp_limiter(phibar, u0, u1, nu)


def interface_flux(order: int, mp: int, pp: int, alpha: float, nu: float, u) -> float:
    u = _stencil(u)
    return _load().vpo_interface_flux(order, mp, pp, alpha, nu,
                                      ctypes.c_void_p(u.ctypes.data + 3 * 8))


def shift_split(s: float):
    n = ctypes.c_long()
    z = ctypes.c_double()
    _load().vpo_shift_split(s, ctypes.byref(n), ctypes.byref(z))
    return n.value, z.value


def advect_line(line, s: float, *, order: int = 7, mp: int = 1, pp: int = 1,
                alpha: float = 4.0, bc: int = BC_PERIODIC) -> np.ndarray:
    """One SL-MPP step of a 1D line by a shift of s cells; returns a new array."""
    out = _f64(line).copy()
    _load().vpo_advect_line(order, mp, pp, alpha, bc, out.size, _p(out), 1, s)
    return out


def rk_line(line, cnu: float, *, mp: int = 1, pp: int = 1, alpha: float = 4.0,
            bc: int = BC_PERIODIC) -> np.ndarray:
    """One RK-MPP5 step (Sec. 2.1.1, Eqs. 8-10) of a 1D line with CFL number
    cnu = c dt / dx (|cnu| < 1/2); returns a new array."""
    out = _f64(line).copy()
    if _load().vpo_rk_mpp5_line(mp, pp, alpha, bc, out.size, _p(out), 1, cnu) != 0:
        raise ValueError("RK-MPP5 needs |c dt / dx| < 1/2")
    return out


# ---- sweeps, moments, Poisson, diagnostics --------------------------------

def _check_f(g: Grid, f: np.ndarray) -> np.ndarray:
    if f.dtype != np.float64 or not f.flags.c_contiguous or f.size != g.NX * g.NV:
        raise ValueError("f must be a C-contiguous float64 array of NX*NV cells")
    return f


def drift_sweep(g: Grid, f: np.ndarray, dim: int, dt: float) -> None:
    """In-place advection along x_dim at speed v_dim (Eq. 4)."""
    if _load().vpo_drift_sweep(ctypes.byref(g), _p(_check_f(g, f)), dim, dt) != 0:
        raise ValueError("bad drift sweep arguments")


def kick_sweep(g: Grid, f: np.ndarray, dim: int, dt: float, accel_dim) -> None:
    """In-place advection along v_dim with acceleration accel_dim[x] (Eq. 5)."""
    a = _f64(accel_dim)
    if a.size != g.NX:
        raise ValueError("accel_dim must hold NX values")
    if _load().vpo_kick_sweep(ctypes.byref(g), _p(_check_f(g, f)), dim, dt, _p(a)) != 0:
        raise ValueError("bad kick sweep arguments")


def drift_unsplit(g: Grid, f: np.ndarray, dt: float) -> None:
    """In-place unsplit advection in physical space (Test-1d, reading R23):
    f <- f + sum_d (A_d f - f), every A_d (the drift_sweep along x_d) applied
    to the same f."""
    if _load().vpo_drift_unsplit(ctypes.byref(g), _p(_check_f(g, f)), dt) != 0:
        raise ValueError("bad unsplit drift arguments")


def drift_sweep_rk(g: Grid, f: np.ndarray, dim: int, dt: float) -> None:
    """drift_sweep with RK-MPP5 lines (every |v dt / dx| < 1/2)."""
    if _load().vpo_drift_sweep_rk(ctypes.byref(g), _p(_check_f(g, f)), dim, dt) != 0:
        raise ValueError("bad RK drift sweep (|v dt / dx| must stay below 1/2)")


def kick_sweep_rk(g: Grid, f: np.ndarray, dim: int, dt: float, accel_dim) -> None:
    """kick_sweep with RK-MPP5 lines (every |a dt / dv| < 1/2)."""
    a = _f64(accel_dim)
    if a.size != g.NX:
        raise ValueError("accel_dim must hold NX values")
    if _load().vpo_kick_sweep_rk(ctypes.byref(g), _p(_check_f(g, f)), dim, dt, _p(a)) != 0:
        raise ValueError("bad RK kick sweep (|a dt / dv| must stay below 1/2)")


def density_moment(g: Grid, f: np.ndarray) -> np.ndarray:
    rho = np.empty(g.NX)
    _load().vpo_density_moment(ctypes.byref(g), _p(_check_f(g, f)), _p(rho))
    return rho


def poisson_solve(g: Grid, rho) -> tuple:
    """Returns (phi[NX], accel[dx, NX]) for the grid's Poisson settings."""
    rho = _f64(rho)
    phi = np.empty(g.NX)
    acc = np.empty(g.dx * g.NX)
    if _load().vpo_poisson_solve(ctypes.byref(g), _p(rho), _p(phi), _p(acc)) != 0:
        raise ValueError("unsupported Poisson configuration")
    return phi, acc.reshape(g.dx, g.NX)


def field(g: Grid, f: np.ndarray) -> tuple:
    rho = density_moment(g, f)
    phi, acc = poisson_solve(g, rho)
    return rho, phi, acc


def diagnostics(g: Grid, f: np.ndarray, mode: int = 1) -> dict:
    rho, phi, acc = field(g, f)
    out = np.empty(NDIAG)
    _load().vpo_diagnostics(ctypes.byref(g), _p(_check_f(g, f)), _p(rho), _p(phi),
                            _p(_f64(acc)), mode, _p(out))
    return dict(zip(DIAG_NAMES, out.tolist()))


def step(g: Grid, f: np.ndarray, dt: float, nsteps: int, accel: np.ndarray, *,
         split: int = SPLIT_KDK, mode: int = 1, diag: bool = False):
    """nsteps Strang steps in place (Sec. 2.4, Eq. 55). accel: (dx, NX), updated.

    Returns an (nsteps, NDIAG) array of diagnostics when diag is true."""
    if accel.dtype != np.float64 or not accel.flags.c_contiguous or accel.size != g.dx * g.NX:
        raise ValueError("accel must be a C-contiguous float64 (dx, NX) array")
    d = np.empty((nsteps, NDIAG)) if diag else None
    rc = _load().vpo_step(ctypes.byref(g), _p(_check_f(g, f)), dt, split, nsteps, _p(accel),
                          mode, _p(d) if d is not None else None)
    if rc != 0:
        raise ValueError("bad step arguments")
    return d


def init_f(g: Grid, kind: int, params) -> np.ndarray:
    p = _f64(params)
    f = np.empty(g.NX * g.NV)
    if _load().vpo_init_f(ctypes.byref(g), kind, _p(p), p.size, _p(f)) != 0:
        raise ValueError("bad initial-condition arguments")
    return f


def cfl_dt(g: Grid, nu: float, accel=None) -> float:
    a = _f64(accel) if accel is not None else None
    return _load().vpo_cfl_dt(ctypes.byref(g), nu, _p(a) if a is not None else None)


def dft(x, sign: int = -1) -> np.ndarray:
    """Plain O(n^2) DFT of a 1D complex sequence (Eq. C4 convention)."""
    x = np.asarray(x, dtype=np.complex128)
    re = np.ascontiguousarray(x.real)
    im = np.ascontiguousarray(x.imag)
    base = np.zeros(1, dtype=np.int64)
    _load().vpo_dft_lines(x.size, 1, _p(base), 1, _p(re), _p(im), sign)
    return re + 1j * im

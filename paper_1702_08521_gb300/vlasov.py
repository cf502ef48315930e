"""Thin ctypes binding of the C ABI in include/vlasov.h (csrc/libvlasov.so).

Functions keep the C names (``vp_create``, ``vp_drift_sweep``, ...) and only
marshal arguments: torch tensors are passed as raw device pointers, a torch
CUDA stream as its ``cudaStream_t``.  Every step of the method runs in the
CUDA library; there is no Python or CPU fallback.  If the library cannot be
loaded, the first call raises ``RuntimeError``.

``Simulation`` is a small convenience owner of a context plus the tensors it
needs (f, acceleration), built on the same calls.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

VP_OK, VP_EINVAL, VP_ECUDA, VP_ENOMEM, VP_ETIMEOUT, VP_ENONFINITE, VP_ENOTSUP, VP_ECFL = 0, -1, -2, -3, -4, -5, -6, -7
VP_F32, VP_F64 = 0, 1
VP_BC_PERIODIC, VP_BC_OUTFLOW = 0, 1
VP_POIS_PERIODIC, VP_POIS_ISOLATED = 0, 1
VP_SPLIT_KDK, VP_SPLIT_DKD = 0, 1
VP_SCHEME_SL, VP_SCHEME_RK = 0, 1
VP_IC_LANDAU, VP_IC_TWOSTREAM, VP_IC_PLUMMER, VP_IC_ADVECT, VP_IC_SPHERE = 0, 1, 2, 3, 4
VP_NDIAG = 9
VP_OPT_SWEEP_IMPL, VP_OPT_AUTOTUNE, VP_OPT_WAIT_LIMIT = 1, 2, 3
DIAG_NAMES = ("mass", "ke", "fe", "pe", "min_f", "max_f", "mode_amp", "l1", "l2")

_lock = threading.Lock()
_lib = None


class VpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"vlasov error {code}: {msg}")
        self.code = code


class vp_grid(ctypes.Structure):
    _fields_ = [
        ("dx", ctypes.c_int), ("dv", ctypes.c_int),
        ("nx", ctypes.c_int * 3), ("nv", ctypes.c_int * 3),
        ("xlo", ctypes.c_double * 3), ("xhi", ctypes.c_double * 3),
        ("vlo", ctypes.c_double * 3), ("vhi", ctypes.c_double * 3),
        ("xbc", ctypes.c_int), ("order", ctypes.c_int), ("mp", ctypes.c_int),
        ("pp", ctypes.c_int), ("alpha", ctypes.c_double), ("precision", ctypes.c_int),
        ("poisson", ctypes.c_int), ("pois_order", ctypes.c_int),
        ("coupling", ctypes.c_double), ("rho_bg", ctypes.c_double),
        ("scheme", ctypes.c_int),
    ]


class vp_run_desc(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int), ("nx", ctypes.c_int * 2), ("nv", ctypes.c_int * 2),
        ("xlo", ctypes.c_double * 2), ("xhi", ctypes.c_double * 2),
        ("vlo", ctypes.c_double * 2), ("vhi", ctypes.c_double * 2),
        ("coupling", ctypes.c_double), ("rho_bg", ctypes.c_double), ("pois_order", ctypes.c_int),
    ]


class vp_diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in DIAG_NAMES]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libvlasov.so (building it first if it is absent or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            try:
                path = _build.build()
            except RuntimeError as e:
                if not os.path.exists(path):
                    raise RuntimeError(f"libvlasov.so is missing and could not be built: {e}") from e
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        GP = ctypes.POINTER(vp_grid)
        sig = {
            "vp_create": (I, [GP, P, ctypes.POINTER(P)]),
            "vp_destroy": (None, [P]),
            "vp_last_error": (ctypes.c_char_p, [P]),
            "vp_num_cells": (LL, [P]),
            "vp_elem_size": (I, [P]),
            "vp_launch_count": (LL, [P]),
            "vp_bind_f": (I, [P, P]),
            "vp_init_f": (I, [P, I, P, I]),
            "vp_upload_f": (I, [P, P, ctypes.c_size_t]),
            "vp_download_f": (I, [P, P, ctypes.c_size_t]),
            "vp_host_alloc": (I, [ctypes.c_size_t, ctypes.POINTER(P)]),
            "vp_host_free": (I, [P]),
            "vp_drift_sweep": (I, [P, I, D]),
            "vp_drift_unsplit": (I, [P, D, I, P]),
            "vp_kick_sweep": (I, [P, I, D, P]),
            "vp_density_moment": (I, [P, P]),
            "vp_poisson_solve": (I, [P, P, P, P]),
            "vp_diagnostics": (I, [P, I, ctypes.POINTER(vp_diag)]),
            "vp_step": (I, [P, D, I, I, P, I, P]),
            "vp_sync": (I, [P]),
            "vp_set_option": (I, [P, I, LL]),
            "vp_get_tuning": (I, [P, I, I, P]),
            "vp_poisson_periodic_noalloc": (I, [GP, P, P, P, P]),
            "vp_ensemble_create": (I, [P, I, I, P, ctypes.POINTER(P)]),
            "vp_ensemble_destroy": (None, [P]),
            "vp_ensemble_last_error": (ctypes.c_char_p, [P]),
            "vp_ensemble_num_cells": (LL, [P]),
            "vp_ensemble_run_layout": (I, [P, I, P, P]),
            "vp_ensemble_bind": (I, [P, P]),
            "vp_ensemble_init_run": (I, [P, I, I, P, I]),
            "vp_ensemble_field": (I, [P]),
            "vp_ensemble_accel": (I, [P, P]),
            "vp_ensemble_set_tiles": (I, [P, I, I, I]),
            "vp_ensemble_get_tiles": (I, [P, P]),
            "vp_ensemble_set_flat_vote": (I, [P, I]),
            "vp_ensemble_get_flat_vote": (I, [P, P]),
            "vp_ensemble_autotune": (I, [P, D]),
            "vp_ensemble_step": (I, [P, D, I]),
            "vp_ensemble_sync": (I, [P]),
            "vp_ensemble_set_wait_limit": (I, [P, LL]),
            "vp_ensemble_launch_count": (LL, [P]),
            "vp_learned_sweep": (I, [P, I, I, D, P, P, I, P]),
            "vp_learned_step": (I, [P, D, I, I, P, P, I, P]),
            "vp_fine_flux": (I, [P, I, I, D, P, I, P]),
            "vp_fluxnet_line_map": (I, [GP, GP, I, I, I, P, P, P]),
            "vp_group_mean": (I, [P, LL, I, P, I, D, P, P]),
            "vp_pair_coefs": (I, [P, P, P, LL, D, P, P, P]),
            "vp_restrict_velocity": (I, [P, P, LL, I, I, I, I, P]),
            "vp_make_samples": (I, [P, I, I, D, P, P, D, P, P, P]),
            "vp_net_grad": (I, [P, P, P, LL, I, P, P, P, P]),
            "vp_net_adam": (I, [P, P, P, P, I, ctypes.c_float, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(t) -> ctypes.c_void_p:
    """Device (or host) pointer of a tensor / integer address / None."""
    if t is None:
        return None
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if isinstance(t, HostBuffer):
        return ctypes.c_void_p(t.ptr)
    return ctypes.c_void_p(t.data_ptr())


def _check(ctx, rc: int) -> None:
    if rc != VP_OK:
        msg = load().vp_last_error(ctx).decode() if ctx else ""
        raise VpError(rc, msg)


def make_grid(dims: int, nx, nv, xlo, xhi, vlo, vhi, *, xbc: int = VP_BC_PERIODIC,
              order: int = 7, mp: int = 1, pp: int = 1, alpha: float = 4.0,
              precision: int = VP_F32, poisson: int = VP_POIS_PERIODIC, pois_order: int = 6,
              coupling: float = -1.0, rho_bg: float = 1.0, scheme: int = 0, **_ignored) -> vp_grid:
    g = vp_grid()
    g.dx = g.dv = dims
    for d in range(dims):
        g.nx[d], g.nv[d] = int(nx[d]), int(nv[d])
        g.xlo[d], g.xhi[d] = float(xlo[d]), float(xhi[d])
        g.vlo[d], g.vhi[d] = float(vlo[d]), float(vhi[d])
    g.xbc, g.order, g.mp, g.pp, g.alpha = xbc, order, mp, pp, float(alpha)
    g.precision, g.poisson, g.pois_order = precision, poisson, pois_order
    g.coupling, g.rho_bg = float(coupling), float(rho_bg)
    g.scheme = int(scheme)
    return g


# ---- the C calls, same names ---------------------------------------------------

def vp_create(grid: vp_grid, stream=None) -> ctypes.c_void_p:
    """stream: a torch.cuda.Stream, an integer cudaStream_t or None (default stream)."""
    lib = load()
    h = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
    out = ctypes.c_void_p()
    rc = lib.vp_create(ctypes.byref(grid), ctypes.c_void_p(h), ctypes.byref(out))
    if rc != VP_OK:
        raise VpError(rc, "vp_create failed (see stderr)")
    return out


def vp_destroy(ctx) -> None:
    load().vp_destroy(ctx)


def vp_last_error(ctx) -> str:
    return load().vp_last_error(ctx).decode()


def vp_num_cells(ctx) -> int:
    return int(load().vp_num_cells(ctx))


def vp_elem_size(ctx) -> int:
    return int(load().vp_elem_size(ctx))


def vp_launch_count(ctx) -> int:
    return int(load().vp_launch_count(ctx))


def vp_bind_f(ctx, f) -> None:
    _check(ctx, load().vp_bind_f(ctx, _ptr(f)))


def vp_init_f(ctx, kind: int, params) -> None:
    arr = (ctypes.c_double * len(params))(*[float(p) for p in params])
    _check(ctx, load().vp_init_f(ctx, kind, ctypes.cast(arr, ctypes.c_void_p), len(params)))


def vp_upload_f(ctx, host, nbytes: int) -> None:
    _check(ctx, load().vp_upload_f(ctx, _ptr(host), nbytes))


def vp_download_f(ctx, host, nbytes: int) -> None:
    _check(ctx, load().vp_download_f(ctx, _ptr(host), nbytes))


class HostBuffer:
    """Page-locked host memory on transparent huge pages (vp_host_alloc), for
    vp_upload_f / vp_download_f; `ptr` is its address, `array(dtype)` a numpy
    view of it.  Freed by close() or when collected."""

    def __init__(self, nbytes: int):
        p = ctypes.c_void_p()
        rc = load().vp_host_alloc(nbytes, ctypes.byref(p))
        if rc != VP_OK:
            raise VpError(rc, f"vp_host_alloc({nbytes}) failed")
        self.ptr, self.nbytes = p.value, nbytes

    def array(self, dtype=np.float32) -> np.ndarray:
        buf = (ctypes.c_char * self.nbytes).from_address(self.ptr)
        return np.frombuffer(buf, dtype=dtype)

    def close(self) -> None:
        if self.ptr:
            load().vp_host_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vp_drift_sweep(ctx, dim: int, dt: float) -> None:
    _check(ctx, load().vp_drift_sweep(ctx, dim, dt))


def vp_drift_unsplit(ctx, dt: float, nsteps: int, scratch) -> None:
    _check(ctx, load().vp_drift_unsplit(ctx, dt, nsteps, _ptr(scratch)))


def vp_kick_sweep(ctx, dim: int, dt: float, accel) -> None:
    _check(ctx, load().vp_kick_sweep(ctx, dim, dt, _ptr(accel)))


def vp_density_moment(ctx, rho) -> None:
    _check(ctx, load().vp_density_moment(ctx, _ptr(rho)))


def vp_poisson_solve(ctx, rho, phi, accel) -> None:
    _check(ctx, load().vp_poisson_solve(ctx, _ptr(rho), _ptr(phi), _ptr(accel)))


def vp_diagnostics(ctx, mode: int = 1) -> dict:
    d = vp_diag()
    _check(ctx, load().vp_diagnostics(ctx, mode, ctypes.byref(d)))
    return {n: getattr(d, n) for n in DIAG_NAMES}


def vp_step(ctx, dt: float, split: int, nsteps: int, accel, mode: int = 1, diag=None) -> None:
    _check(ctx, load().vp_step(ctx, dt, split, nsteps, _ptr(accel), mode, _ptr(diag)))


def vp_sync(ctx) -> None:
    _check(ctx, load().vp_sync(ctx))


def vp_set_option(ctx, option: int, value: int) -> None:
    _check(ctx, load().vp_set_option(ctx, option, value))


def vp_get_tuning(ctx, kick: int, dim: int) -> dict:
    out = (ctypes.c_int * 4)()
    _check(ctx, load().vp_get_tuning(ctx, kick, dim, ctypes.cast(out, ctypes.c_void_p)))
    return {"impl": out[0], "tile": out[1], "segments": out[2], "ctas_per_sm": out[3]}


VP_NOALLOC_MAX_POINTS = 262144


def vp_poisson_periodic_noalloc(grid: vp_grid, stream, rho, phi, accel) -> int:
    """Allocation-free periodic Poisson solve (returns the VP_* status code)."""
    h = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
    return int(load().vp_poisson_periodic_noalloc(ctypes.byref(grid), ctypes.c_void_p(h), _ptr(rho),
                                                  _ptr(phi), _ptr(accel)))


# ---- batched ensembles -----------------------------------------------------------

def _echeck(ens, rc: int) -> None:
    if rc != VP_OK:
        raise VpError(rc, load().vp_ensemble_last_error(ens).decode() if ens else "")


def make_run(dims: int, nx, nv, xlo, xhi, vlo, vhi, coupling: float = -1.0, rho_bg: float = 1.0,
             pois_order: int = 6, **_ignored) -> vp_run_desc:
    r = vp_run_desc()
    r.dims = dims
    for d in range(dims):
        r.nx[d], r.nv[d] = int(nx[d]), int(nv[d])
        r.xlo[d], r.xhi[d], r.vlo[d], r.vhi[d] = float(xlo[d]), float(xhi[d]), float(vlo[d]), float(vhi[d])
    r.coupling, r.rho_bg, r.pois_order = float(coupling), float(rho_bg), int(pois_order)
    return r


def vp_ensemble_create(runs, order: int = 7, stream=None):
    arr = (vp_run_desc * len(runs))(*runs)
    h = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
    out = ctypes.c_void_p()
    rc = load().vp_ensemble_create(ctypes.cast(arr, ctypes.c_void_p), len(runs), order, ctypes.c_void_p(h),
                                   ctypes.byref(out))
    if rc != VP_OK:
        raise VpError(rc, "vp_ensemble_create failed")
    return out


def vp_ensemble_destroy(ens) -> None:
    load().vp_ensemble_destroy(ens)


def vp_ensemble_num_cells(ens) -> int:
    return int(load().vp_ensemble_num_cells(ens))


def vp_ensemble_run_layout(ens, run: int):
    f = ctypes.c_longlong()
    a = ctypes.c_longlong()
    _echeck(ens, load().vp_ensemble_run_layout(ens, run, ctypes.byref(f), ctypes.byref(a)))
    return f.value, a.value


def vp_ensemble_bind(ens, pool) -> None:
    _echeck(ens, load().vp_ensemble_bind(ens, _ptr(pool)))


def vp_ensemble_init_run(ens, run: int, kind: int, params) -> None:
    arr = (ctypes.c_double * len(params))(*[float(p) for p in params])
    _echeck(ens, load().vp_ensemble_init_run(ens, run, kind, ctypes.cast(arr, ctypes.c_void_p), len(params)))


def vp_ensemble_field(ens) -> None:
    _echeck(ens, load().vp_ensemble_field(ens))


def vp_ensemble_accel(ens) -> int:
    p = ctypes.c_void_p()
    _echeck(ens, load().vp_ensemble_accel(ens, ctypes.byref(p)))
    return p.value


def vp_ensemble_set_tiles(ens, W: int, R: int, ctas_per_sm: int = 0) -> None:
    _echeck(ens, load().vp_ensemble_set_tiles(ens, W, R, ctas_per_sm))


def vp_ensemble_get_tiles(ens) -> dict:
    out = (ctypes.c_int * 3)()
    _echeck(ens, load().vp_ensemble_get_tiles(ens, ctypes.cast(out, ctypes.c_void_p)))
    return {"W": out[0], "R": out[1], "ctas_per_sm": out[2]}


def vp_ensemble_set_flat_vote(ens, on: int) -> None:
    _echeck(ens, load().vp_ensemble_set_flat_vote(ens, on))


def vp_ensemble_get_flat_vote(ens) -> int:
    out = ctypes.c_int()
    _echeck(ens, load().vp_ensemble_get_flat_vote(ens, ctypes.byref(out)))
    return out.value


def vp_ensemble_autotune(ens, dt: float) -> None:
    _echeck(ens, load().vp_ensemble_autotune(ens, dt))


def vp_ensemble_step(ens, dt: float, nsteps: int) -> None:
    _echeck(ens, load().vp_ensemble_step(ens, dt, nsteps))


def vp_ensemble_sync(ens) -> None:
    _echeck(ens, load().vp_ensemble_sync(ens))


def vp_ensemble_set_wait_limit(ens, iterations: int) -> None:
    _echeck(ens, load().vp_ensemble_set_wait_limit(ens, int(iterations)))


def vp_ensemble_launch_count(ens) -> int:
    return int(load().vp_ensemble_launch_count(ens))


# ---- learned flux correction -----------------------------------------------------

VP_NET_NPARAM = 2977


def _sh(stream):
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0))


def _rc(rc: int, what: str) -> None:
    if rc != VP_OK:
        raise VpError(rc, what)


def vp_learned_sweep(ctx, kick: int, dim: int, dt: float, accel, wts, use_net: int = 1, f_snap=None) -> None:
    _check(ctx, load().vp_learned_sweep(ctx, kick, dim, dt, _ptr(accel), _ptr(wts), use_net, _ptr(f_snap)))


def vp_learned_step(ctx, dt: float, split: int, nsteps: int, accel, wts, mode: int = 1, diag=None) -> None:
    _check(ctx, load().vp_learned_step(ctx, dt, split, nsteps, _ptr(accel), _ptr(wts), mode, _ptr(diag)))


def vp_fine_flux(ctx, kick: int, dim: int, dt: float, accel, every: int, G) -> None:
    _check(ctx, load().vp_fine_flux(ctx, kick, dim, dt, _ptr(accel), every, _ptr(G)))


def vp_fluxnet_line_map(fine: vp_grid, coarse: vp_grid, factor: int, kick: int, dim: int):
    """Returns (map as a list of ints, n_coarse_lines, group)."""
    n = ctypes.c_longlong()
    g = ctypes.c_int()
    L = load()
    _rc(L.vp_fluxnet_line_map(ctypes.byref(fine), ctypes.byref(coarse), factor, kick, dim, None,
                              ctypes.byref(n), ctypes.byref(g)), "line map")
    arr = (ctypes.c_longlong * (n.value * g.value))()
    _rc(L.vp_fluxnet_line_map(ctypes.byref(fine), ctypes.byref(coarse), factor, kick, dim,
                              ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(n), ctypes.byref(g)), "line map")
    return list(arr), n.value, g.value


def vp_group_mean(G_fine, n_coarse_lines: int, nout: int, map_dev, group: int, scale: float, G_coarse,
                  stream=None) -> None:
    _rc(load().vp_group_mean(_ptr(G_fine), n_coarse_lines, nout, _ptr(map_dev), group, scale,
                             _ptr(G_coarse), _sh(stream)), "group mean")


def vp_pair_coefs(sc, li, ri, n: int, importance: float, coef, weight=None, stream=None) -> None:
    _rc(load().vp_pair_coefs(_ptr(sc), _ptr(li), _ptr(ri), int(n), float(importance), _ptr(coef),
                             _ptr(weight), _sh(stream)), "pair coefficients")


def vp_restrict_velocity(f_fine, f_coarse, NX: int, nf1: int, nf2: int, factor1: int, factor2: int,
                         stream=None) -> None:
    _rc(load().vp_restrict_velocity(_ptr(f_fine), _ptr(f_coarse), NX, nf1, nf2, factor1, factor2,
                                    _sh(stream)), "restrict")


def vp_make_samples(ctx, kick: int, dim: int, dt: float, accel, Gc, zmin: float, X, y, scale=None) -> None:
    _check(ctx, load().vp_make_samples(ctx, kick, dim, dt, _ptr(accel), _ptr(Gc), zmin, _ptr(X), _ptr(y),
                                       _ptr(scale)))


def vp_net_grad(X, y, nsamp: int, wts, grad, loss, stream=None, coef=None, group: int = 1) -> None:
    _rc(load().vp_net_grad(_ptr(X), _ptr(y), _ptr(coef), nsamp, group, _ptr(wts), _ptr(grad), _ptr(loss),
                           _sh(stream)),
        "net grad")


def vp_net_adam(wts, m, v, grad, step: int, lr: float, stream=None) -> None:
    _rc(load().vp_net_adam(_ptr(wts), _ptr(m), _ptr(v), _ptr(grad), step, lr, _sh(stream)), "adam")


# ---- convenience owner -----------------------------------------------------------

class Simulation:
    """A context plus its device tensors (torch is used for memory and streams)."""

    def __init__(self, grid: dict, precision: int = VP_F32, stream=None, device: str = "cuda"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the Vlasov library needs a CUDA device")
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.grid = make_grid(**{**grid, "precision": precision})
        self.ctx = vp_create(self.grid, self.stream)
        self.dims = grid["dims"]
        self.shape = tuple(grid["nx"]) + tuple(grid["nv"])
        self.NX = 1
        for n in grid["nx"]:
            self.NX *= int(n)
        dtype = torch.float32 if precision == VP_F32 else torch.float64
        self.f = torch.empty(vp_num_cells(self.ctx), dtype=dtype, device=device)
        self.accel = torch.zeros(self.dims * self.NX, dtype=torch.float64, device=device)
        self.rho = torch.zeros(self.NX, dtype=torch.float64, device=device)
        self.phi = torch.zeros(self.NX, dtype=torch.float64, device=device)
        vp_bind_f(self.ctx, self.f)

    def init(self, kind: int, params) -> None:
        vp_init_f(self.ctx, kind, params)

    def upload(self, f_host) -> None:
        """Copy a host array / tensor into f (blocking)."""
        t = self.torch.as_tensor(f_host).to(self.f.dtype).contiguous()
        with self.torch.cuda.stream(self.stream):
            self.f.copy_(t.reshape(-1), non_blocking=False)
        self.stream.synchronize()

    def field(self) -> None:
        vp_density_moment(self.ctx, self.rho)
        vp_poisson_solve(self.ctx, self.rho, self.phi, self.accel)

    def step(self, dt: float, nsteps: int, split: int = VP_SPLIT_KDK, mode: int = 1, diag=None):
        vp_step(self.ctx, dt, split, nsteps, self.accel, mode, diag)

    def learned_step(self, dt: float, nsteps: int, wts, split: int = VP_SPLIT_KDK, mode: int = 1, diag=None):
        vp_learned_step(self.ctx, dt, split, nsteps, self.accel, wts, mode, diag)

    def diagnostics(self, mode: int = 1) -> dict:
        return vp_diagnostics(self.ctx, mode)

    def sync(self) -> None:
        vp_sync(self.ctx)

    def close(self) -> None:
        if self.ctx:
            vp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""FP64 reference of the learned flux correction (test infrastructure only).

Not part of the paper: the learned correction is an addition to the method.
It is restated here in plain numpy, in double precision, so that the GPU
training and inference kernels can be checked against it.

Network (per interface of a spatial sweep; upwind-ordered stencil u_{-3..4} of
the line, u_0 = upwind cell; u+_k / u-_k: the same cells on the lines of the
neighbouring velocity cells of the sweep's axis, + on the side of larger |v|):
    s    = max_k |u_k| + 1e-30
    x    = [(u_k - u_0) / s for k = -3..4]
         + [(u+_k - u-_k) / (2 s) for k = -3..4]
         + [(u+_k + u-_k - 2 u_k) / (2 s) for k = -3..4] + [nu]   (25 features)
    h1   = relu(W1 x  + b1)      W1: 32 x 25
    h2   = relu(W2 h1 + b2)      W2: 32 x 32
    h3   = relu(W3 h2 + b3)      W3: 32 x 32
    g    = w4 . h3 + b4          w4: 32
    M    = nu * MP(Phi_CSL) + s * g   (mass through the interface)
    M    = clamp(M, nu f_min, nu f_max)  (optional: the MP bounds of Appendix A
                                       again, in mass form)
    M    = PP(M)                     (Eqs. 15-23 with 2 nu Phi written as 2 M)
    f'_i = f_{i-N} - (M_out - M_in)  (flux form, Eq. 49 with nu Phi -> M)
Weights and every matrix input (x, h1, h2, h3) are rounded to bfloat16 as on
the tensor cores; sums are exact here (FP64) and FP32 on the GPU.  Target of
g at an interface: y = (M_target - nu MP(Phi_CSL)) / s.  Training loss: the
mean over cells of r^2, r = (s_r (g_r - y_r) - s_l (g_l - y_l)) / max(s_l, s_r)
over the cell's right / left interface, i.e. the error of the cell update
(loss_and_grad with group = 2); group = 1 gives the per-interface error.
The backward pass treats the bfloat16 rounding as the identity.

learned_line() is the whole learned SL update of one line in this form.  It
is written in masses so that it needs no division by nu: at nu = 0 (an
integer shift) the MP bounds in mass form have zero width, every mass is 0
and the update is the exact shift of the line.
"""
from __future__ import annotations

import numpy as np

from . import BC_PERIODIC, csl_flux, mp_bounds, mp_constraint, shift_split

HIDDEN = 32
NFEAT = 25
SHAPES = {"W1": (HIDDEN, NFEAT), "b1": (HIDDEN,), "W2": (HIDDEN, HIDDEN), "b2": (HIDDEN,),
          "W3": (HIDDEN, HIDDEN), "b3": (HIDDEN,), "w4": (HIDDEN,), "b4": (1,)}
ORDER = ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4")


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if np.any(nan):
        out[nan] = np.nan
    return out


def features(u, up, um, nu) -> tuple:
    """u, up, um: (B, 8) upwind-ordered stencils u_{-3..4} of the line and of
    its velocity neighbours (+: larger |v|); nu: (B,). Returns (X, s): the
    stencil relative to u_0, the velocity difference and the velocity
    curvature at the 8 cells, all over s = max |u|, and nu."""
    u = np.asarray(u, dtype=np.float64)
    up = np.asarray(up, dtype=np.float64)
    um = np.asarray(um, dtype=np.float64)
    s = np.abs(u).max(axis=1) + 1e-30
    dv = (up - um) / (2.0 * s[:, None])
    cv = (up + um - 2.0 * u) / (2.0 * s[:, None])
    X = np.concatenate([(u - u[:, 3:4]) / s[:, None], dv, cv, np.asarray(nu, dtype=np.float64)[:, None]],
                       axis=1)
    return X, s


def init_params(seed: int = 0) -> dict:
    rng = np.random.default_rng(seed)
    p = {}
    for k, shp in SHAPES.items():
        if k.startswith("W") or k == "w4":
            fan_in = shp[-1] if len(shp) == 2 else HIDDEN
            p[k] = rng.normal(0.0, np.sqrt(2.0 / fan_in), size=shp) * (0.1 if k == "w4" else 1.0)
        else:
            p[k] = np.zeros(shp)
    return p


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel() for k in ORDER])


def unpack(v) -> dict:
    v = np.asarray(v, dtype=np.float64)
    p, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        p[k] = v[o:o + n].reshape(SHAPES[k])
        o += n
    return p


def forward(p: dict, X, *, round_bf16: bool = True):
    """g (B,) and the cache for backward."""
    q = (lambda a: bf16(a)) if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    W1, W2, W3, w4 = q(p["W1"]), q(p["W2"]), q(p["W3"]), q(p["w4"])
    x0 = q(X)
    z1 = x0 @ W1.T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    x1 = q(h1)
    z2 = x1 @ W2.T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    x2 = q(h2)
    z3 = x2 @ W3.T + p["b3"]
    h3 = np.maximum(z3, 0.0)
    x3 = q(h3)
    g = x3 @ w4 + p["b4"][0]
    return g, (x0, z1, x1, z2, x2, z3, x3, W1, W2, W3, w4)


def loss_and_grad(p: dict, X, y, *, round_bf16: bool = True, coef=None, group: int = 1):
    """Loss and its gradient (dict) over the batch.  Samples form consecutive
    groups of `group` with residual r = sum_k a_k (g_k - y_k) (a = coef, or
    all 1); the loss is the mean of r^2 over groups (group 1, no coef: the
    mean squared error)."""
    g, (x0, z1, x1, z2, x2, z3, x3, W1, W2, W3, w4) = forward(p, X, round_bf16=round_bf16)
    B = len(y)
    a = np.ones(B) if coef is None else np.asarray(coef, dtype=np.float64)
    term = a * (g - np.asarray(y, dtype=np.float64))
    r = term.reshape(-1, group).sum(axis=1)
    loss = float(np.mean(r * r))
    dg = 2.0 * np.repeat(r, group) * a / (B // group)
    grads = {"w4": x3.T @ dg, "b4": np.array([dg.sum()])}
    dh3 = np.outer(dg, w4) * (z3 > 0)
    grads["W3"] = dh3.T @ x2
    grads["b3"] = dh3.sum(axis=0)
    dh2 = (dh3 @ W3) * (z2 > 0)
    grads["W2"] = dh2.T @ x1
    grads["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (z1 > 0)
    grads["W1"] = dh1.T @ x0
    grads["b1"] = dh1.sum(axis=0)
    return loss, grads


def pp_mass(M: float, u0: float, u1: float, nu: float) -> float:
    """PP flux limiter of Sec. 2.1.1 (Eqs. 15-23) in mass form: the interface
    carries M = nu Phi out of the upwind cell u0 into u1.  Both halves of the
    update, u0 - 2 M and u1 + 2 M, must stay >= 0; where one would not, M is
    blended towards the upwind mass nu u0 by theta (same reading of theta
    under rounding as the oracle's flux-form limiter: (1 - 8 eps) when it
    binds, clamped to [0, 1], 0 for a non-positive denominator)."""
    u_plus, u_up_plus = u0 - 2.0 * M, u0 - 2.0 * nu * u0
    u_minus, u_up_minus = u1 + 2.0 * M, u1 + 2.0 * nu * u0
    th_plus = th_minus = 1.0
    binds = False
    if u_plus < 0.0:
        den = u_up_plus - u_plus
        th_plus = u_up_plus / den if den > 0.0 else 0.0
        binds = True
    if u_minus < 0.0:
        den = u_up_minus - u_minus
        th_minus = u_up_minus / den if den > 0.0 else 0.0
        binds = True
    th = min(th_plus, th_minus)
    if binds:
        th *= 1.0 - 8.0 * 2.0 ** -53
    th = min(max(th, 0.0), 1.0)
    return th * M + (1.0 - th) * (nu * u0)


def learned_line(line, up_line, um_line, s: float, p: dict, bc: int = BC_PERIODIC,
                 alpha: float = 4.0, mp_bound: bool = False) -> np.ndarray:
    """One learned SL update of a spatial line by a shift of s cells.

    line: the line's cells; up_line / um_line: the same cells on the lines of
    the neighbouring velocity cells (+: the side of larger |v|), zeros where
    the velocity grid ends.  Steps, per interface of the shifted line (upwind
    cell q, stencil u_{-3..4} in upwind order): the CSL7 flux (Sec. 2.1.2),
    the MP constraint (Appendix A), the network correction s g, with mp_bound
    the MP bounds on the total in mass form, the PP limiter in mass form; then
    the flux-form update of every cell (Eq. 49).  Shift decomposition s = N + zeta as in the
    plain sweep (nearest integer N, nu = |zeta|, direction sign zeta)."""
    line = np.asarray(line, dtype=np.float64)
    L = line.size
    n_int, zeta = shift_split(s)
    sg = -1 if zeta < 0 else 1
    nu = abs(zeta)

    def val(a, k):
        if bc == BC_PERIODIC:
            return float(a[k % L])
        return float(a[k]) if 0 <= k < L else 0.0

    def mass(q):
        idx = [q + sg * (k - 3) for k in range(8)]
        u = np.array([val(line, i) for i in idx])
        up = np.array([val(up_line, i) for i in idx])
        um = np.array([val(um_line, i) for i in idx])
        phi = mp_constraint(csl_flux(7, nu, u[:7]), u[:7], alpha)
        X, sc = features(u[None, :], up[None, :], um[None, :], np.array([nu]))
        M = nu * phi + sc[0] * forward(p, X)[0][0]
        if mp_bound:
            fmin, fmax = mp_bounds(u[:7], alpha)
            M = min(max(M, nu * fmin), nu * fmax)
        return pp_mass(M, u[3], u[4], nu)

    out = np.empty(L)
    for i in range(L):
        q = i - n_int
        out[i] = val(line, q) - (mass(q) - mass(q - sg))
    return out

"""Seeded synthetic inputs and workload descriptions.

This module is shared by the tests, the benchmark and the oracle-driven
checks.  It holds NONE of the method's arithmetic: only grid sizes, boxes,
time steps, initial-condition parameters, and seeded random arrays that are
handed unchanged to both the CUDA path and the CPU oracle.

Workloads (all synthetic, analytic initial conditions of the paper or of
standard plasma/stellar-dynamics tests, no external data):

* ``landau_linear``     1D1V linear Landau damping, Nx=64, Nv=128, FP64, MP5+PP,
                        dt=0.1, 200 steps (Sec. 3.3 with Nv doubled).
* ``landau_nonlinear``  1D1V nonlinear Landau (alpha=0.5, k=0.5), Nx=256, Nv=1024,
                        v in [-8, 8], MP7+PP, FP32, dt=0.05, 1000 steps.
* ``two_stream``        1D1V two-stream, same grid and scheme.
* ``plummer``           3D3V Plummer sphere (G=M=a=1), 32^3 x 64^3, x in [-4,4]^3,
                        v in [-1.5,1.5]^3, isolated Poisson, MP7+PP, FP32, DKD,
                        dt=0.05, 50 steps.
* ``ensemble``          512 uneven 1D1V runs + 8 2D2V Landau runs, parameters drawn
                        from numpy PCG64(seed=1702).
* ``jeans_slab``        1D1V self-gravitating slab of Sec. 3.2 (Test-2), k/k_J = 0.5
                        (unstable) or 1.1 (damped), G = mean density = L = 1.
* ``uniform_sphere``    3D3V collapse of a uniform sphere (Sec. 3.4, Test-4),
                        64^3 x 32^3, G = M = R = 1.
"""
from __future__ import annotations

import math

import numpy as np

TWO_PI = 2.0 * math.pi

# boundary / Poisson / split / IC codes (plain integers; both sides define their own)
BC_PERIODIC, BC_OUTFLOW = 0, 1
POIS_PERIODIC, POIS_ISOLATED = 0, 1
SPLIT_KDK, SPLIT_DKD = 0, 1
IC_LANDAU, IC_TWOSTREAM, IC_PLUMMER, IC_ADVECT, IC_SPHERE = 0, 1, 2, 3, 4


def _grid(dims, nx, nv, xlo, xhi, vlo, vhi, **kw) -> dict:
    g = dict(dims=dims, nx=list(nx), nv=list(nv), xlo=list(xlo), xhi=list(xhi),
             vlo=list(vlo), vhi=list(vhi), xbc=BC_PERIODIC, order=7, mp=1, pp=1, alpha=4.0,
             poisson=POIS_PERIODIC, pois_order=6, coupling=-1.0, rho_bg=1.0)
    g.update(kw)
    return g


def landau_linear() -> dict:
    L = 4.0 * math.pi
    return dict(name="landau_linear_1d1v_64x128",
                grid=_grid(1, [64], [128], [0.0], [L], [-6.0], [6.0], order=5),
                ic=(IC_LANDAU, [0.01, 0.5, 0.0, 0.0, 1.0, 1.0]),
                dt=0.1, steps=200, split=SPLIT_KDK, precision="f64", mode=1)


def landau_nonlinear(nx: int = 256, nv: int = 1024) -> dict:
    L = 4.0 * math.pi
    return dict(name=f"landau_nonlinear_1d1v_{nx}x{nv}",
                grid=_grid(1, [nx], [nv], [0.0], [L], [-8.0], [8.0], order=7),
                ic=(IC_LANDAU, [0.5, 0.5, 0.0, 0.0, 1.0, 1.0]),
                dt=0.05, steps=1000, split=SPLIT_KDK, precision="f32", mode=1)


def two_stream(nx: int = 256, nv: int = 1024) -> dict:
    L = 4.0 * math.pi
    return dict(name=f"two_stream_1d1v_{nx}x{nv}",
                grid=_grid(1, [nx], [nv], [0.0], [L], [-8.0], [8.0], order=7),
                ic=(IC_TWOSTREAM, [0.05, 0.5]),
                dt=0.05, steps=1000, split=SPLIT_KDK, precision="f32", mode=1)


def plummer(nx: int = 32, nv: int = 64, box: float = 4.0, vbox: float = 1.5) -> dict:
    return dict(name=f"plummer_3d3v_{nx}^3x{nv}^3",
                grid=_grid(3, [nx] * 3, [nv] * 3, [-box] * 3, [box] * 3, [-vbox] * 3, [vbox] * 3,
                           order=7, xbc=BC_OUTFLOW, poisson=POIS_ISOLATED, pois_order=6,
                           coupling=4.0 * math.pi, rho_bg=0.0),
                ic=(IC_PLUMMER, [1.0, 1.0, 1.0]),
                dt=0.05, steps=50, split=SPLIT_DKD, precision="f32", mode=1)


def uniform_sphere(nx: int = 64, nv: int = 32, precision: str = "f32") -> dict:
    """Sec. 3.4 (Test-4): a uniform sphere of mass M and radius 2R (Eq. 77,
    sigma^2 = G M / (20 R), virial ratio 0.5) in units G = M = R = 1, so that
    T = (R^3 / G M)^(1/2) = 1 and V = R / T = 1; box [-3R, 3R]^3 x [-3V, 3V]^3
    with outgoing boundaries in x and v and the isolated Poisson solver;
    SL-MPP7, DKD, the time step of Sec. 2.4 (nu = 0.2) each step, to t = 8T."""
    return dict(name=f"uniform_sphere_3d3v_{nx}^3x{nv}^3",
                grid=_grid(3, [nx] * 3, [nv] * 3, [-3.0] * 3, [3.0] * 3, [-3.0] * 3, [3.0] * 3,
                           order=7, xbc=BC_OUTFLOW, poisson=POIS_ISOLATED, pois_order=6,
                           coupling=4.0 * math.pi, rho_bg=0.0),
                ic=(IC_SPHERE, [1.0, 1.0, 1.0]),
                t_end=8.0, nu=0.2, split=SPLIT_DKD, precision=precision, mode=1)


def jeans_slab(ratio: float = 0.5, n: int = 64, amp: float | None = None, precision: str = "f32") -> dict:
    """Sec. 3.2 (Test-2): the slab of Eq. 69 in units G = mean density = L = 1,
    so that the dynamical time T = (G rho)^(-1/2) = 1 and V = L / T = 1.
    k = 4 pi / L; sigma from k / k_J = ratio with k_J = (4 pi G rho)^(1/2) / sigma
    (Eq. 71); A = 0.01 and v in [-V, V] for ratio < 1, A = 0.1 and v in
    [-2V, 2V] otherwise; periodic x, zero-inflow v, gravity (S = 4 pi G) with
    the mean density as background.  The runs end at t = 4T with the time step
    of Sec. 2.4 (nu = 0.2, Eqs. 56-58) taken each step."""
    k = 4.0 * math.pi
    sigma = ratio * math.sqrt(4.0 * math.pi) / k
    vmax = 1.0 if ratio < 1.0 else 2.0
    a = amp if amp is not None else (0.01 if ratio < 1.0 else 0.1)
    return dict(name=f"jeans_slab_1d1v_{n}x{n}_k/kJ={ratio}",
                grid=_grid(1, [n], [n], [0.0], [1.0], [-vmax], [vmax], order=7,
                           coupling=4.0 * math.pi, rho_bg=1.0),
                ic=(IC_LANDAU, [a, k, 0.0, 0.0, sigma, 1.0]),
                k=k, sigma=sigma, t_end=4.0, nu=0.2, split=SPLIT_KDK, precision=precision, mode=2)


def advect_1d(n: int, shape: int, order: int = 7, mp: int = 1, pp: int = 1,
              speed: float = 1.0) -> dict:
    """Test-1 style pure advection: one velocity cell centred on `speed`."""
    return dict(name=f"advect_1d_{n}",
                grid=_grid(1, [n], [1], [0.0], [1.0], [speed - 0.5], [speed + 0.5], order=order,
                           mp=mp, pp=pp),
                ic=(IC_ADVECT, [float(shape)]))


def advect_2d(n: int, shape: int, order: int = 7, mp: int = 1, pp: int = 1, n2: int = None,
              nv: int = 1) -> dict:
    """Test-1d two-dimensional advection: n x n2 cells on the unit square,
    periodic, velocity range [0.5, 1.5] x [0, 1] in nv x nv cells (nv = 1: the
    single velocity (c_x, c_y) = (1, 0.5) of the paper; nv = 2: four such
    problems at once, (c_x, c_y) in {0.75, 1.25} x {0.25, 0.75})."""
    n2 = n if n2 is None else n2
    tag = "" if nv == 1 else f"x{nv}x{nv}"
    return dict(name=f"advect_2d_{n}x{n2}{tag}",
                grid=_grid(2, [n, n2], [nv, nv], [0.0, 0.0], [1.0, 1.0], [0.5, 0.0], [1.5, 1.0], order=order,
                           mp=mp, pp=pp),
                ic=(IC_ADVECT, [float(shape)]))


def random_f(shape, seed: int, *, zeros: float = 0.3, dtype=np.float64) -> np.ndarray:
    """Non-negative structured noise: a smooth bump field times a random mask
    with exact zeros, plus small-scale noise (stresses MP and PP branches)."""
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    base = rng.random(n) ** rng.choice([1.0, 2.0, 4.0])
    mask = rng.random(n) >= zeros
    out = (base * mask).reshape(shape)
    return out.astype(dtype)


def random_accel(nx_total: int, dims: int, seed: int, amax: float) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-amax, amax, size=(dims, nx_total))


def ensemble_draws(n1d: int = 512, n2d: int = 8, seed: int = 1702) -> list:
    """Parameter draws of the batched ensemble: kind, Nx, Nv, k, alpha."""
    rng = np.random.Generator(np.random.PCG64(seed))
    runs = []
    for _ in range(n1d):
        kind = "landau" if rng.random() < 0.5 else "two_stream"
        nx = int(rng.choice([32, 64, 128, 256]))
        nv = int(rng.choice([64, 128, 256, 512]))
        k = float(rng.uniform(0.3, 0.6))
        alpha = float(rng.uniform(0.001, 0.5))
        vmax = 6.0 if kind == "landau" else 8.0
        runs.append(dict(kind=kind, dims=1, nx=[nx], nv=[nv], k=[k], alpha=alpha,
                         xlo=[0.0], xhi=[TWO_PI / k], vlo=[-vmax], vhi=[vmax]))
    for _ in range(n2d):
        alpha = float(rng.uniform(0.001, 0.5))
        runs.append(dict(kind="landau", dims=2, nx=[64, 64], nv=[64, 64], k=[0.5, 0.5],
                         alpha=alpha, xlo=[0.0, 0.0], xhi=[TWO_PI / 0.5] * 2,
                         vlo=[-6.0, -6.0], vhi=[6.0, 6.0]))
    return runs

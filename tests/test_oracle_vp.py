"""Pins of the oracle's Vlasov-Poisson composition (Sec. 2.4, Sec. 3.3).

Pins: the Landau damping rate and frequency from the kinetic dispersion
relation (solved here with scipy's Faddeeva function, independent of the
oracle) against the printed gamma = 0.153; moments of the analytic initial
conditions; conservation of mass and total energy; the Plummer density.
"""
import math

import numpy as np
import pytest
from scipy.optimize import fsolve
from scipy.special import erfc, wofz

import oracle as O
from paper_1702_08521_gb300 import inputs


def landau_root(k: float):
    """Root of 1 + (1 + xi Z(xi)) / k^2 = 0, xi = omega / (k sqrt 2),
    Z(xi) = i sqrt(pi) w(xi) (Maxwellian electrons, unit thermal speed)."""
    def eq(p):
        om = p[0] + 1j * p[1]
        xi = om / (k * math.sqrt(2.0))
        Z = 1j * math.sqrt(math.pi) * wofz(xi)
        d = 1 + (1 + xi * Z) / k ** 2
        return [d.real, d.imag]
    wr, wi = fsolve(eq, [1.4, -0.15], xtol=1e-13)
    return wr, wi


def fit_damping(t, amp, t0=2.0, t1=18.0):
    """Local maxima of ln|E_k| in [t0, t1] (three-point parabolic refinement),
    least-squares slope -> gamma; pi / mean spacing of maxima -> omega."""
    la = np.log(amp)
    pk_t, pk_v = [], []
    for i in range(1, len(t) - 1):
        if la[i] > la[i - 1] and la[i] >= la[i + 1] and t0 <= t[i] <= t1:
            y0, y1, y2 = la[i - 1], la[i], la[i + 1]
            den = y0 - 2 * y1 + y2
            d = 0.5 * (y0 - y2) / den if den != 0 else 0.0
            h = t[1] - t[0]
            pk_t.append(t[i] + d * h)
            pk_v.append(y1 - 0.25 * (y0 - y2) * d)
    pk_t, pk_v = np.array(pk_t), np.array(pk_v)
    gamma = np.polyfit(pk_t, pk_v, 1)[0]
    omega = math.pi / np.mean(np.diff(pk_t))
    return gamma, omega, pk_t


def test_landau_root_matches_printed_rate():
    wr, wi = landau_root(0.5)
    assert abs(wi + 0.153) < 1e-3          # gamma = 0.153 (Sec. 3.3)
    assert wr == pytest.approx(1.4156, abs=1e-4)


def _setup(cfg):
    g = O.grid(**cfg["grid"])
    kind, params = cfg["ic"]
    f = O.init_f(g, kind, params)
    return g, f


def test_landau_initial_moments():
    cfg = inputs.landau_linear()
    g, f = _setup(cfg)
    rho = O.density_moment(g, f)
    x = g.x_centres(0)
    # what is left besides the truncation of the velocity box at |v| = 6 is
    # the midpoint rule's end correction h^2/24 |f'(6)| * 2 ~ 3e-11
    trunc = 1.0 - erfc(6.0 / math.sqrt(2.0))
    assert np.allclose(rho, trunc * (1 + 0.01 * np.cos(0.5 * x)), rtol=1e-10, atol=0)
    d = O.diagnostics(g, f)
    L = 4 * math.pi
    assert d["mass"] == pytest.approx(L * trunc, rel=1e-10)
    # <v^2> = sigma^2 = 1 minus the tail beyond |v| = 6
    ke_tail = 6.0 * math.exp(-18.0) / math.sqrt(2 * math.pi) * 2
    assert d["ke"] == pytest.approx(0.5 * L * (trunc - ke_tail), rel=1e-9)
    # E field of rho = 1 + A cos kx: a = A sin(kx)/k -> mode amplitude A/k
    assert d["mode_amp"] == pytest.approx(0.01 / 0.5, rel=1e-4)


@pytest.mark.slow
def test_linear_landau_damping_rate_and_frequency():
    """Config: Nx = 64, Nv = 128, v in [-6, 6], MP5+PP, dt = 0.1, 200 steps.
    The measured damping rate and frequency of |E_{k=0.5}| match the
    dispersion relation (gamma within 3 %, omega within 1 %)."""
    cfg = inputs.landau_linear()
    g, f = _setup(cfg)
    _, _, acc = O.field(g, f)
    acc = np.ascontiguousarray(acc)
    d0 = O.diagnostics(g, f)
    diag = O.step(g, f, cfg["dt"], cfg["steps"], acc, split=cfg["split"], mode=1, diag=True)
    t = cfg["dt"] * np.arange(0, cfg["steps"] + 1)
    amp = np.concatenate([[d0["mode_amp"]], diag[:, 6]])
    gamma, omega, pk = fit_damping(t, amp)
    wr, wi = landau_root(0.5)
    assert len(pk) >= 6
    assert gamma == pytest.approx(wi, rel=0.03), (gamma, wi)
    assert omega == pytest.approx(wr, rel=0.01), (omega, wr)
    # mass is conserved up to what leaves through the velocity boundary
    # (f(|v| = 6) ~ 6e-9: zero-inflow velocity boundaries), f >= 0, and total
    # energy is conserved to the splitting error
    assert np.all(np.abs(diag[:, 0] / d0["mass"] - 1) < 1e-9)
    assert diag[:, 4].min() >= 0.0
    e_tot = diag[:, 1] + diag[:, 2]
    assert np.abs(e_tot / (d0["ke"] + d0["fe"]) - 1).max() < 1e-5


def test_two_stream_initial_moments():
    cfg = inputs.two_stream(nx=32, nv=256)
    g, f = _setup(cfg)
    rho = O.density_moment(g, f)
    x = g.x_centres(0)
    # int v^2 e^{-v^2/2}/sqrt(2 pi) dv = 1 (truncation at |v| = 8 negligible)
    assert np.allclose(rho, 1 + 0.05 * np.cos(0.5 * x), rtol=1e-9, atol=0)


def test_nonlinear_landau_short_run_invariants():
    """Nonlinear Landau (alpha = 0.5) on a reduced grid: mass conserved,
    f >= 0, energy conserved to the splitting error."""
    cfg = inputs.landau_nonlinear(nx=32, nv=128)
    g, f = _setup(cfg)
    _, _, acc = O.field(g, f)
    acc = np.ascontiguousarray(acc)
    d0 = O.diagnostics(g, f)
    diag = O.step(g, f, cfg["dt"], 100, acc, split=cfg["split"], diag=True)
    assert np.abs(diag[:, 0] / d0["mass"] - 1).max() < 1e-12
    assert diag[:, 4].min() >= 0.0
    e = diag[:, 1] + diag[:, 2]
    assert np.abs(e / (d0["ke"] + d0["fe"]) - 1).max() < 5e-3


def test_kdk_and_dkd_agree_to_second_order():
    cfg = inputs.landau_nonlinear(nx=32, nv=64)
    g, f0 = _setup(cfg)
    errs = []
    for dt in (0.1, 0.05):
        out = []
        for split in (O.SPLIT_KDK, O.SPLIT_DKD):
            f = f0.copy()
            _, _, acc = O.field(g, f)
            acc = np.ascontiguousarray(acc)
            O.step(g, f, dt, int(round(1.0 / dt)), acc, split=split)
            out.append(f)
        errs.append(np.abs(out[0] - out[1]).sum() / np.abs(out[0]).sum())
    assert errs[1] < errs[0] / 3.0  # ~ dt^2


def test_plummer_density_at_t0():
    """The isotropic Plummer DF integrates to rho(r) = 3/(4 pi) (1 + r^2)^-5/2
    (G = M = a = 1) up to the velocity-grid quadrature error."""
    cfg = inputs.plummer(nx=8, nv=24)
    g, f = _setup(cfg)
    rho = O.density_moment(g, f)
    c = g.x_centres(0)
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    r2 = (X ** 2 + Y ** 2 + Z ** 2).ravel()
    want = 3 / (4 * math.pi) * (1 + r2) ** -2.5
    core = r2 < 2.0
    assert np.max(np.abs(rho[core] / want[core] - 1)) < 0.05
    assert f.min() >= 0.0

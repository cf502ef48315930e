"""Pins of the oracle's line update and 1D/2D advection (Test-1 of Sec. 3.1).

Pins: exact integer shifts, translation and mirror invariance, the
telescoping mass identity of the flux form (Eq. 49), the paper's Test-1a/1c
statements, and measured orders of accuracy on smooth translation.
"""
import numpy as np
import pytest

import oracle as O
from paper_1702_08521_gb300 import inputs


def test_shift_split_rounds_half_away_from_zero():
    assert O.shift_split(2.5) == (3, -0.5)
    assert O.shift_split(-2.5) == (-3, 0.5)
    assert O.shift_split(0.49) == (0, 0.49)
    n, z = O.shift_split(7.3)
    assert n == 7 and z == pytest.approx(0.3, abs=1e-15)


@pytest.mark.parametrize("order", [5, 7])
def test_integer_shift_is_an_exact_copy(order):
    rng = np.random.default_rng(2)
    f = rng.random(37)
    for n in (-40, -3, 0, 1, 5, 36):
        assert np.array_equal(O.advect_line(f, float(n), order=order), np.roll(f, n))
        out = O.advect_line(f, float(n), order=order, bc=O.BC_OUTFLOW)
        want = np.zeros_like(f)
        if n >= 0:
            want[n:] = f[:len(f) - n] if n < len(f) else []
        else:
            want[:n] = f[-n:]
        assert np.array_equal(out, want)


def test_integer_plus_fraction_is_roll_of_fraction():
    """Periodic: advecting by N + zeta equals rolling the zeta-advected line
    by N, bit for bit (the integer part is an exact copy)."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        f = rng.random(29)
        n = int(rng.integers(-9, 10))
        s = n + rng.uniform(-0.5, 0.5)
        z = s - n  # exact: the fractional part the split will see
        a = O.advect_line(f, s)
        b = np.roll(O.advect_line(f, z), n)
        assert np.array_equal(a, b)


def test_mirror_symmetry():
    """c < 0 is the mirror image of c > 0 (Sec. 2.1)."""
    rng = np.random.default_rng(4)
    for _ in range(100):
        f = rng.random(32) * (rng.random(32) < 0.8)
        s = rng.uniform(-3, 3)
        order = int(rng.choice([5, 7]))
        bc = int(rng.integers(0, 2))
        a = O.advect_line(f, s, order=order, bc=bc)
        b = O.advect_line(f[::-1].copy(), -s, order=order, bc=bc)[::-1]
        assert np.array_equal(a, b)


def test_mass_is_conserved_by_the_flux_form():
    """Periodic: sum f' = sum f up to rounding (telescoping fluxes, Eq. 49)."""
    rng = np.random.default_rng(8)
    for _ in range(200):
        L = int(rng.integers(8, 200))
        f = rng.random(L) * (rng.random(L) < 0.8)
        g = O.advect_line(f, rng.uniform(-6, 6), order=int(rng.choice([5, 7])))
        assert abs(g.sum() - f.sum()) <= 4 * L * 2.0 ** -53 * np.abs(f).sum()


def test_outflow_mass_budget_closes():
    """Zero-inflow boundaries: the mass lost equals nu times the flux through
    the boundary interface (computed here from the line's own fluxes)."""
    rng = np.random.default_rng(9)
    for _ in range(50):
        L = 24
        f = rng.random(L)
        s = rng.uniform(0.05, 0.5)
        g = O.advect_line(f, s, order=7, bc=O.BC_OUTFLOW)
        pad = np.concatenate([np.zeros(4), f, np.zeros(4)])
        j = 4 + L - 1  # upwind cell of the right boundary interface
        flux = O.interface_flux(7, 1, 1, 4.0, s, pad[j - 3:j + 4])
        flux_in = O.interface_flux(7, 1, 1, 4.0, s, pad[4 - 1 - 3:4 - 1 + 4])
        assert g.sum() == pytest.approx(f.sum() - s * (flux - flux_in), rel=1e-13, abs=1e-14)


def _advect_run(n, shape, order, mp, pp, nu, T, offset=0.0):
    g = O.grid(**inputs.advect_1d(n, shape, order=order, mp=mp, pp=pp)["grid"])
    f = O.init_f(g, O.IC_ADVECT, [shape]) + offset
    dt = nu / n
    steps = int(round(T / dt))
    for _ in range(steps):
        O.drift_sweep(g, f, 0, dt)
    xe = (g.x_centres(0) - steps * dt) % 1.0
    if shape == 0:
        ex = ((xe >= 0.25) & (xe <= 0.75)).astype(float)
    elif shape == 1:
        ex = 1.0 + np.sin(2 * np.pi * xe)
    else:
        ex = np.sin(4 * np.pi * xe) ** 4
    ex = ex + offset
    return np.abs(f - ex).sum() / np.abs(ex).sum(), f


@pytest.mark.parametrize("order,slope", [(5, 4.5), (7, 6.3)])
def test_order_of_accuracy_smooth_translation(order, slope):
    """Test-1b: 1 + sin(2 pi x), nu = 0.2, t = 1; SL-MP5 ~5th and SL-MP7 ~7th
    order in L1 (Eq. 61).  With PP on, the same orders on the profile lifted
    by 0.1 (see the reading on Test-1b: with a minimum exactly at zero the PP
    condition binds even for the exact flux)."""
    for pp, off in ((0, 0.0), (1, 0.1)):
        errs = [_advect_run(n, 1, order, 1, pp, 0.2, 1.0, off)[0] for n in (16, 32, 64, 128)]
        slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        floor = 1e-12
        for e_hi, e_lo, s in zip(errs[:-1], errs[1:], slopes):
            if e_lo > floor:
                assert s >= slope, (order, pp, errs, slopes)


def test_large_shifts_match_small_shift_error():
    """With s = 3 + 1/4 per step (dyadic, so the split is exact) the result is
    the s = 1/4 result rolled by 3 cells per step, bit for bit."""
    n = 64
    g = O.grid(**inputs.advect_1d(n, 1)["grid"])
    f0 = O.init_f(g, O.IC_ADVECT, [1.0])
    a = f0.copy()
    b = f0.copy()
    for _ in range(50):
        O.drift_sweep(g, a, 0, 0.25 / n)
        O.drift_sweep(g, b, 0, 3.25 / n)
    assert np.array_equal(np.roll(a, 150), b)


def test_rectangle_stays_within_bounds():
    """Test-1a: N = 64, t = 8, nu = 0.2; no over/undershoot (Sec. 3.1.1)."""
    for order in (5, 7):
        err, f = _advect_run(64, 0, order, 1, 1, 0.2, 8.0)
        assert f.min() >= 0.0 and f.max() <= 1.0
        assert err < 0.2


def test_rectangle_first_order_convergence():
    """Test-1a: errors scale about as N^-1 (Sec. 3.1.1)."""
    errs = [_advect_run(n, 0, 7, 1, 1, 0.2, 1.0)[0] for n in (32, 64, 128, 256)]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 0.5) and np.all(slopes < 1.5), slopes


def test_quartic_sine_positivity():
    """Test-1c: sin^4(4 pi x), N = 64, t = 8: SL-MP5 without PP goes negative,
    SL-MPP5 and SL-MPP7 stay >= 0 (Sec. 3.1.3)."""
    _, f_mp = _advect_run(64, 2, 5, 1, 0, 0.2, 8.0)
    assert f_mp.min() < -1e-3
    for order in (5, 7):
        _, f = _advect_run(64, 2, order, 1, 1, 0.2, 8.0)
        assert f.min() >= 0.0
    e5 = _advect_run(64, 2, 5, 1, 1, 0.2, 8.0)[0]
    e7 = _advect_run(64, 2, 7, 1, 1, 0.2, 8.0)[0]
    assert e7 < e5  # SL-MPP7 reproduces the profile better


def test_quartic_sine_near_fifth_order():
    """Test-1c: SL-MPP5/7 close to fifth order on sin^4 (Sec. 3.1.3)."""
    for order in (5, 7):
        errs = [_advect_run(n, 2, order, 1, 1, 0.2, 1.0)[0] for n in (64, 128, 256)]
        slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        assert slopes[-1] > 3.8, (order, errs, slopes)


def test_two_dimensional_split_advection_order():
    """Test-1d: c = (1, 0.5), split sweeps keep the 1D order on the 2D sine."""
    def run(n, order):
        g = O.grid(2, [n, n], [1, 1], [0, 0], [1, 1], [0.5, 0.0], [1.5, 1.0], order=order, pp=1)
        f = O.init_f(g, O.IC_ADVECT, [1.0]) + 0.1
        dt = 0.2 / n
        steps = int(round(0.5 / dt))
        for _ in range(steps):
            O.drift_sweep(g, f, 1, dt)
            O.drift_sweep(g, f, 0, dt)
        x = g.x_centres(0)[:, None]
        y = g.x_centres(1)[None, :]
        t = steps * dt
        ex = 1.1 + 0.5 * np.sin(2 * np.pi * (x - t)) + 0.5 * np.sin(2 * np.pi * (y - 0.5 * t))
        return np.abs(f.reshape(n, n) - ex).sum() / np.abs(ex).sum()
    for order, slope in ((5, 4.5), (7, 6.0)):
        errs = [run(n, order) for n in (16, 32, 64)]
        slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        assert np.all(slopes >= slope), (order, errs, slopes)


def test_oracle_grid_struct_matches_its_header():
    """oracle.Grid lists vpo_grid's fields (oracle/vp_oracle.h) in order, and
    the IC / boundary codes agree with the header's."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "oracle", "vp_oracle.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} vpo_grid;", src, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            names += [re.sub(r"\[.*\]", "", p).strip() for p in decl.split(None, 1)[1].split(",")]
    assert [f[0] for f in O.Grid._fields_] == names
    defs = {m.group(1): int(m.group(2)) for m in re.finditer(r"^#define\s+VPO_(\w+)\s+(-?\d+)", src, flags=re.M)}
    for n in ("IC_LANDAU", "IC_TWOSTREAM", "IC_PLUMMER", "IC_ADVECT", "IC_SPHERE", "BC_PERIODIC", "BC_OUTFLOW"):
        assert getattr(O, n) == defs[n], n


# ---- unsplit advection (Test-1d, reading R23) --------------------------------

def _g2(n, order=7, n2=None, **kw):
    return O.grid(**{**inputs.advect_2d(n, 1, order=order, n2=n2)["grid"], **kw})


@pytest.mark.parametrize("order", [5, 7])
def test_unsplit_on_product_data_is_the_sum_of_the_1d_increments(order):
    """For f = g(x) h(y) with g, h > 0 every x line is h_j g and every y line
    g_i h, and the SL-MPP update (CSL flux, MP bounds, PP clamp) is positively
    homogeneous, so the unsplit step is h A_x g + g A_y h - g h with A_x, A_y
    the 1D line updates, while a split step would give (A_x g)(A_y h).
    Shifts with integer parts and both signs (c = (1, -0.5) scaled by dt)."""
    n1, n2 = 23, 17
    g = O.grid(2, [n1, n2], [1, 1], [0, 0], [1, 1], [0.5, -1.0], [1.5, 0.0], order=order)
    rng = np.random.default_rng(41)
    gx = 0.2 + rng.random(n1) ** 2
    hy = 0.2 + rng.random(n2) ** 2
    gx[5:8] = gx[5]  # a flat run (the MP bounds collapse there)
    for dt in (0.37 / n1, 2.71 / n1):
        f = np.outer(gx, hy).ravel().copy()
        O.drift_unsplit(g, f, dt)
        ax = O.advect_line(gx, 1.0 * dt * n1, order=order)
        ay = O.advect_line(hy, -0.5 * dt * n2, order=order)
        want = np.outer(ax, hy) + np.outer(gx, ay) - np.outer(gx, hy)
        assert np.allclose(f.reshape(n1, n2), want, rtol=0, atol=1e-14)
        split = np.outer(ax, ay)
        assert np.abs(split - want).max() > 1e-4  # the cross term the unsplit step drops


def test_unsplit_equals_split_on_sum_separable_data():
    """f = 1 + (sin 2 pi x + sin 2 pi y) / 2 (Eq. 66): an x line is a 1D profile
    plus a constant, which the x update carries unchanged, so unsplit and split
    steps both give A_x g + A_y h (to rounding) -- the reason the paper sees
    the same errors with both on its Test-1d profiles."""
    g = _g2(24)
    f0 = O.init_f(g, O.IC_ADVECT, [1.0])
    fu, fs = f0.copy(), f0.copy()
    dt = 0.02 / 24
    for _ in range(30):
        O.drift_unsplit(g, fu, dt)
        O.drift_sweep(g, fs, 1, dt)
        O.drift_sweep(g, fs, 0, dt)
    assert np.abs(fu - fs).max() < 1e-13
    assert np.abs(fu - f0).max() > 1e-2


@pytest.mark.parametrize("order,slope", [(5, 4.8), (7, 6.8)])
def test_unsplit_sine_order_at_the_papers_cfl(order, slope):
    """Test-1d with the unsplit method at nu = 0.02 (Sec. 3.1): the 2D sine keeps
    the scheme's spatial order, N = 16, 32, 64 to t = 0.5."""
    def err(n):
        g = _g2(n, order)
        f = O.init_f(g, O.IC_ADVECT, [1.0])
        dt = 0.02 / n
        steps = int(round(0.5 / dt))
        for _ in range(steps):
            O.drift_unsplit(g, f, dt)
        x, y, t = g.x_centres(0)[:, None], g.x_centres(1)[None, :], steps * dt
        ex = 1 + 0.5 * np.sin(2 * np.pi * (x - t)) + 0.5 * np.sin(2 * np.pi * (y - 0.5 * t))
        return np.abs(f.reshape(n, n) - ex).sum() / np.abs(ex).sum()
    errs = [err(n) for n in (16, 32, 64)]
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes >= slope), (errs, slopes)


def test_unsplit_rectangle_needs_the_small_cfl():
    """Test-1d rectangle (Eq. 65), N = 32, t = 0.25: at nu = 0.02 the unsplit
    method stays within [0, 1]; at nu = 0.45 it overshoots and goes negative
    (the paper keeps nu below 0.1 for the unsplit runs), while the split
    sweeps stay non-negative at any nu."""
    def run(nu, unsplit):
        g = _g2(32)
        f = O.init_f(g, O.IC_ADVECT, [0.0])
        dt = nu / 32
        for _ in range(int(round(0.25 / dt))):
            if unsplit:
                O.drift_unsplit(g, f, dt)
            else:
                O.drift_sweep(g, f, 1, dt)
                O.drift_sweep(g, f, 0, dt)
        return f
    f = run(0.02, True)
    assert f.min() >= 0.0 and f.max() <= 1.0
    f = run(0.45, True)
    assert f.min() < -1e-5 and f.max() > 1.05
    assert run(0.45, False).min() >= 0.0


def test_unsplit_conserves_mass_and_constants():
    """Periodic space: sum f is kept to rounding (each increment is a
    difference of interface masses); a constant stays constant.  2D2V and 3D
    space with several velocities per axis."""
    rng = np.random.default_rng(5)
    for dims, nx, nv in ((2, [12, 9], [4, 3]), (3, [6, 5, 7], [2, 3, 2])):
        g = O.grid(dims, nx, nv, [0.0] * dims, [1.0] * dims, [-2.0] * dims, [2.0] * dims, order=7)
        f = inputs.random_f(g.NX * g.NV, seed=9)
        m0 = f.sum()
        for dt in (0.013, 0.21):
            O.drift_unsplit(g, f, dt)
        assert abs(f.sum() - m0) < 1e-12 * m0
        c = np.full(g.NX * g.NV, 0.375)
        O.drift_unsplit(g, c, 0.3)
        assert np.all(c == 0.375)
    g = O.grid(2, [8, 8], [2, 2], [0, 0], [1, 1], [-1, -1], [1, 1], xbc=O.BC_OUTFLOW)
    f = rng.random(g.NX * g.NV)
    m0 = f.sum()
    O.drift_unsplit(g, f, 0.05)
    assert f.sum() < m0  # zero inflow: mass leaves through the boundaries

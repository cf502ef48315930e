"""Pins of the oracle's RK-MPP5 scheme (Sec. 2.1.1, Eqs. 8-10), the variant
the paper compares SL-MPP5 against.

Pins: third-order convergence to the exact solution of smooth periodic
advection at a fixed CFL number (fifth order in space, third in time; a wrong
coefficient of Eq. 8 or of Eq. 10 breaks consistency); constants kept
exactly; mass conserved; the mirror image of a line advected the other way;
no new maximum with the MP constraint; f >= 0 with the PP limiter where the
unlimited scheme goes negative; the CFL bound |nu| < 1/2.
"""
import math

import numpy as np
import pytest

import oracle as O


def _cell_avg_sine(n, shift=0.0):
    """Exact cell averages of 1 + 0.5 sin(2 pi (x - shift)) on [0, 1)."""
    h = 1.0 / n
    xl = np.arange(n) * h - shift
    return 1.0 + 0.5 * (np.cos(2 * np.pi * xl) - np.cos(2 * np.pi * (xl + h))) / (2 * np.pi * h)


def _advect(n, nu, periods=1.0, mp=0, pp=0):
    u = _cell_avg_sine(n)
    steps = int(round(periods * n / nu))
    for _ in range(steps):
        u = O.rk_line(u, nu, mp=mp, pp=pp)
    return u, _cell_avg_sine(n, steps * nu / n)


def test_rk_mpp5_converges_at_third_order_on_smooth_data():
    errs = []
    for n in (32, 64, 128):
        u, ex = _advect(n, 0.2)
        errs.append(np.abs(u - ex).mean())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    # above 3 while the fifth-order spatial error still counts, falling
    # towards the third order of the time integration (measured 3.97, 3.40)
    assert all(2.8 < p < 4.5 for p in orders), (errs, orders)
    assert orders[1] < orders[0] and orders[1] < 3.6, orders
    # the MP constraint keeps the accuracy of a smooth profile (extrema included)
    u, ex = _advect(128, 0.2, mp=1)
    assert np.abs(u - ex).mean() < 2 * errs[-1]


def test_rk_small_cfl_exposes_fifth_order_space():
    """At nu = 0.02 the time error (nu h)^3 is small: the spatial order shows."""
    errs = []
    for n in (16, 32):
        u, ex = _advect(n, 0.02, periods=0.25)
        errs.append(np.abs(u - ex).mean())
    assert math.log2(errs[0] / errs[1]) > 4.3, errs


def test_rk_invariants():
    rng = np.random.default_rng(3)
    u = rng.uniform(0.0, 1.0, 50)
    # constants stay constant (Eq. 8 weights sum to one, Eq. 10 is consistent)
    c = np.full(40, 0.37)
    assert np.array_equal(O.rk_line(c, 0.3), c) or np.abs(O.rk_line(c, 0.3) - c).max() < 1e-15
    # periodic mass conservation
    v = O.rk_line(u, 0.41)
    assert abs(v.sum() - u.sum()) < 1e-13 * u.sum()
    # advecting the reversed line the other way gives the reversed result
    w = O.rk_line(u[::-1].copy(), -0.41)
    assert np.allclose(w[::-1], v, rtol=0, atol=1e-15)


def test_rk_limiters():
    n = 64
    sq = np.where((np.arange(n) >= 16) & (np.arange(n) < 32), 1.0, 0.0)
    u_mp, u_free, u_both = sq.copy(), sq.copy(), sq.copy()
    neg_free = 0.0
    for _ in range(60):
        u_free = O.rk_line(u_free, 0.3, mp=0, pp=0)
        neg_free = min(neg_free, u_free.min())
        u_mp = O.rk_line(u_mp, 0.2, mp=1, pp=0)  # MP bound needs nu <= 1 / (1 + alpha)
        u_both = O.rk_line(u_both, 0.3, mp=1, pp=1)
        assert u_mp.max() <= 1.0 + 1e-14  # monotonicity preserving: no new maximum
        assert u_both.min() >= 0.0
    assert neg_free < -1e-3  # the unlimited scheme overshoots below zero


def test_rk_cfl_bound():
    with pytest.raises(ValueError):
        O.rk_line(np.ones(16), 0.5)
    with pytest.raises(ValueError):
        O.rk_line(np.ones(16), -0.7)

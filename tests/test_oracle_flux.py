"""Pins of the oracle's single-interface functions (CSL flux, MP, PP).

Each pin comes from outside the oracle's own code: the defining integral of
the SL flux (Sec. 2.1.2, Eqs. 26-27) evaluated exactly for polynomials, the
separately printed interface interpolants (Eqs. 8 and 24), special cases of
Appendix A worked by hand, and the positivity claim of Sec. 2.1.1.
"""
import numpy as np
import pytest

import oracle as O


def cell_avgs_of_poly(coef, cells):
    """Cell averages over [j - 1/2, j + 1/2] of sum_k coef[k] x^k (unit cells)."""
    out = []
    for j in cells:
        a, b = j - 0.5, j + 0.5
        out.append(sum(c * (b ** (k + 1) - a ** (k + 1)) / (k + 1) for k, c in enumerate(coef)))
    return np.array(out)


def departure_mean(coef, nu):
    """(1 / nu) * integral of the polynomial over [1/2 - nu, 1/2]: the exact
    SL flux through the interface x = 1/2 (Eq. 27 with Delta x = 1)."""
    a, b = 0.5 - nu, 0.5
    return sum(c * (b ** (k + 1) - a ** (k + 1)) / (k + 1) for k, c in enumerate(coef)) / nu


@pytest.mark.parametrize("order,degree", [(5, 4), (7, 6)])
def test_csl_flux_exact_on_polynomials(order, degree):
    """CSL_p reproduces the exact departure-interval mean for every polynomial
    of degree <= p-1 and every nu: this fixes all p x p coefficients C_j / D_j."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        coef = rng.normal(size=degree + 1)
        nu = rng.uniform(1e-3, 1.0)
        u = cell_avgs_of_poly(coef, range(-3, 4))
        want = departure_mean(coef, nu)
        got = O.csl_flux(order, nu, u)
        assert abs(got - want) <= 1e-12 * (1 + np.abs(u).max()), (order, nu, got, want)


@pytest.mark.parametrize("order,degree", [(5, 5), (7, 7)])
def test_csl_flux_not_exact_one_degree_higher(order, degree):
    """The order is exactly p: degree p data is not reproduced (a test that a
    wider, wrong stencil cannot pass)."""
    coef = [0.0] * degree + [1.0]
    u = cell_avgs_of_poly(coef, range(-3, 4))
    assert abs(O.csl_flux(order, 0.3, u) - departure_mean(coef, 0.3)) > 1e-6


def test_csl_flux_zero_shift_is_printed_interpolant():
    """At zeta -> 0 the flux is the interface value: Eq. (8) for MP5 and
    Eq. (24) for MP7, printed separately from the CSL tables."""
    rng = np.random.default_rng(6)
    for _ in range(100):
        u = rng.normal(size=7)  # u[-3..3]; u[0] = f_{i-1}
        fim4, fim3, fim2, fim1, fi, fip1, fip2 = u
        int5 = (2 * fim3 - 13 * fim2 + 47 * fim1 + 27 * fi - 3 * fip1) / 60.0
        int7 = (-3 * fim4 + 25 * fim3 - 101 * fim2 + 319 * fim1 + 214 * fi - 38 * fip1 + 4 * fip2) / 420.0
        assert O.csl_flux(5, 0.0, u) == pytest.approx(int5, abs=1e-13)
        assert O.csl_flux(7, 0.0, u) == pytest.approx(int7, abs=1e-13)


def test_csl_flux_full_cell_shift_is_upwind_cell():
    """nu = 1: the departure interval is exactly the upwind cell."""
    rng = np.random.default_rng(7)
    for _ in range(100):
        u = rng.normal(size=7)
        assert O.csl_flux(5, 1.0, u) == pytest.approx(u[3], abs=1e-13)
        assert O.csl_flux(7, 1.0, u) == pytest.approx(u[3], abs=1e-13)


# ---- MP constraint, Appendix A -------------------------------------------

def test_mp_local_maximum_clips_to_cell_value():
    """u = (0, 1, 2, 1, 0) around f_i = 2: f* = f_i, the accept test fails and
    steps 4-7 give f_min = f_max = 2 (hand evaluation)."""
    u = np.array([0.0, 0.0, 1.0, 2.0, 1.0, 0.0, 0.0])
    for phi in (2.7, 1.3, -5.0, 2.0):
        assert O.mp_constraint(phi, u) == 2.0


def test_mp_step_gives_upwind_value():
    """A step from 0 to 1 just downwind: every bound collapses to f_i = 0."""
    u = np.array([0.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
    for phi in (0.4, -0.1, 0.9):
        assert O.mp_constraint(phi, u) == 0.0


def test_mp_accepts_interior_value_on_linear_data():
    """Linear data: Phi strictly between f_i and f* = f_{i+1} is kept (step 3)."""
    u = np.arange(7, dtype=float) * 0.5 + 1.0
    for nu in (0.1, 0.3, 0.7):
        phi = O.csl_flux(7, nu, u)
        assert O.mp_constraint(phi, u) == phi


def test_mp_keeps_monotone_profiles_monotone():
    """SL-MP with nu <= 1/(1+alpha) on monotone ramps (random, and stair-cased)
    between plateaus keeps them monotone with no new extrema (the property the
    MP constraint is built for, Sec. 2.1 requirement (i))."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        ramp = np.sort(rng.random(16))
        if rng.random() < 0.5:
            ramp = np.round(ramp * 4) / 4
        f = np.concatenate([np.full(24, ramp[0]), ramp, np.full(24, ramp[-1])])
        order = int(rng.choice([5, 7]))
        s = rng.uniform(0, 0.2) * rng.choice([-1, 1])
        g = f.copy()
        for _ in range(10):
            g = O.advect_line(g, s, order=order, mp=1, pp=int(rng.integers(0, 2)), bc=O.BC_OUTFLOW)
        inner = g[12:-12]
        assert np.all(np.diff(inner) >= -1e-15)
        assert inner.max() <= f.max() + 1e-15 and inner.min() >= f.min() - 1e-15


# ---- PP limiter, Sec. 2.1.1 -----------------------------------------------

def test_pp_inactive_when_both_halves_positive():
    assert O.pp_limiter(0.5, 1.0, 1.0, 0.3) == 0.5


def test_pp_binding_zeroes_the_outflow_half():
    """A flux that would empty the upwind cell is blended so that U^+ = 0 up
    to the safety factor: f_i - 2 nu Phi^ is tiny and non-negative."""
    u0, u1, nu = 0.2, 0.3, 0.4
    ph = O.pp_limiter(5.0, u0, u1, nu)
    uplus = u0 - 2 * nu * ph
    assert 0.0 <= uplus <= 1e-14
    assert u0 <= ph < 5.0


def test_pp_full_upwind_at_half_cfl():
    """nu = 1/2: U^{UP,+} = 0, so a binding limiter returns the upwind value."""
    assert O.pp_limiter(3.0, 1.0, 0.0, 0.5) == 1.0


def test_pp_guarantees_nonnegative_updates_on_random_data():
    """f >= 0 in, f >= 0 out (exactly), for random shifts with integer parts,
    both schemes and both boundary kinds."""
    rng = np.random.default_rng(11)
    for _ in range(1500):
        L = int(rng.integers(8, 40))
        f = rng.random(L) ** rng.choice([1, 4, 8]) * (rng.random(L) < 0.7)
        s = rng.uniform(-5, 5)
        g = O.advect_line(f, s, order=int(rng.choice([5, 7])), mp=1, pp=1,
                          bc=int(rng.integers(0, 2)))
        assert g.min() >= 0.0


def test_exact_flux_violates_pp_condition_near_a_quadratic_zero():
    """Worked example behind the design notes' reading of Test-1b: for
    f = (x - x0)^2 and the cell [x0 - 0.1, x0 + 0.9] at nu = 0.2, even the
    exact SL flux gives U^+ = f_i - 2 nu Phi < 0, so the PP limiter must bind
    at a minimum that touches zero."""
    f_i = (0.9 ** 3 + 0.1 ** 3) / 3.0
    phi = (0.9 ** 3 - 0.7 ** 3) / (3.0 * 0.2)
    assert f_i - 2 * 0.2 * phi < 0.0


# ---- MP constraint, Appendix A steps 4-7 on non-degenerate stencils --------
#
# Stencils are written as (f_{i-2}, f_{i-1}, f_i, f_{i+1}, f_{i+2}) (f_{i-3} is
# not used).  Every value is a binary fraction so that the hand-worked bounds
# below are exact in double precision.

def _stencil5(a, b, c, d, e):
    return np.array([0.0, a, b, c, d, e, 0.0])


def test_mp_md_bound_above_the_downwind_cell():
    """Concave stencil (0, 3, 5, 5.5, 4), alpha = 4:
    step 2: f* = 5 + minmod(0.5, 8) = 5.5, so step 3 keeps only (5, 5.5);
    step 4: d_{i-1} = 0 + 5 - 6 = -1, d_i = 3 + 5.5 - 10 = -1.5,
            d_{i+1} = 5 + 4 - 11 = -2;
            d^M4_{i+1/2} = minmod(-6 + 2, -8 + 1.5, -1.5, -2) = -1.5,
            d^M4_{i-1/2} = minmod(-4 + 1.5, -6 + 1, -1, -1.5) = -1;
    step 5: f^UL = 5 + 4 * 2 = 13, f^AV = 5.25, f^MD = 5.25 + 0.75 = 6,
            f^LC = 5 + 1 - 4/3 = 14/3;
    step 6: f^min = max(min(5, 5.5, 6), min(5, 13, 14/3)) = 5,
            f^max = min(max(5, 5.5, 6), max(5, 13, 14/3)) = 6 (= f^MD).
    So values above f_{i+1} up to f^MD survive (the curvature allowance) and
    6.3 is cut to 6.  Dropping the 1/2 on d^M4 would give f^MD = 6.75."""
    u = _stencil5(0.0, 3.0, 5.0, 5.5, 4.0)
    assert O.mp_bounds(u) == (5.0, 6.0)
    assert O.mp_constraint(6.3, u) == 6.0
    assert O.mp_constraint(5.8, u) == 5.8
    assert O.mp_constraint(4.0, u) == 5.0
    assert O.mp_constraint(5.25, u) == 5.25   # accepted by step 3


def test_mp_md_bound_from_the_4x_minus_y_argument():
    """Convex stencil (4.5, 2.75, 2, 2.25, 6): the smallest argument of the
    d^M4 minmod is 4 d_i - d_{i+1}, not d_i or d_{i+1}.
    step 2: f* = 2 + minmod(0.25, 4 * (-0.75)) = 2: step 3 never keeps phi;
    step 4: d_{i-1} = 4.5 + 2 - 5.5 = 1, d_i = 2.75 + 2.25 - 4 = 1,
            d_{i+1} = 2 + 6 - 4.5 = 3.5;
            d^M4_{i+1/2} = minmod(4 - 3.5, 14 - 1, 1, 3.5) = 0.5,
            d^M4_{i-1/2} = minmod(3, 3, 1, 1) = 1;
    step 5: f^UL = 2 - 3 = -1, f^AV = 2.125, f^MD = 2.125 - 0.25 = 1.875,
            f^LC = 2 - 0.375 + 4/3 = 71/24;
    step 6: f^min = max(min(2, 2.25, 1.875), min(2, -1, 71/24)) = 1.875 (= f^MD),
            f^max = min(max(2, 2.25, 1.875), max(2, -1, 71/24)) = 2.25.
    minmod(d_i, d_{i+1}) = 1 in place of 0.5 would put f^min at 1.625."""
    u = _stencil5(4.5, 2.75, 2.0, 2.25, 6.0)
    assert O.mp_bounds(u) == (1.875, 2.25)
    assert O.mp_constraint(1.5, u) == 1.875
    assert O.mp_constraint(1.9, u) == 1.9
    assert O.mp_constraint(2.5, u) == 2.25


def test_mp_lc_bound_from_the_4y_minus_x_argument():
    """Stencil (11.5, 3, 2, 3, 6): f^LC is the upper bound, with d^M4_{i-1/2}
    from the argument 4 d_i - d_{i-1}.
    step 2: f* = 2 + minmod(1, -4) = 2: step 3 never keeps phi;
    step 4: d_{i-1} = 11.5 + 2 - 6 = 7.5, d_i = 3 + 3 - 4 = 2,
            d_{i+1} = 2 + 6 - 6 = 2;
            d^M4_{i-1/2} = minmod(30 - 2, 8 - 7.5, 7.5, 2) = 0.5,
            d^M4_{i+1/2} = minmod(6, 6, 2, 2) = 2;
    step 5: f^UL = 2 - 4 = -2, f^AV = 2.5, f^MD = 2.5 - 1 = 1.5,
            f^LC = 2 - 0.5 + (4/3) 0.5 = 13/6;
    step 6: f^min = max(min(2, 3, 1.5), min(2, -2, 13/6)) = 1.5 (= f^MD),
            f^max = min(max(2, 3, 1.5), max(2, -2, 13/6)) = 13/6 (= f^LC).
    A 4 in place of 4/3 (f^LC = 3.5) or minmod(d_{i-1}, d_i) = 2 (f^LC = 25/6)
    would leave f^max = 3."""
    u = _stencil5(11.5, 3.0, 2.0, 3.0, 6.0)
    lo, hi = O.mp_bounds(u)
    assert lo == 1.5 and hi == pytest.approx(13.0 / 6.0, abs=4e-16)
    assert O.mp_constraint(2.6, u) == hi
    assert O.mp_constraint(1.0, u) == 1.5
    assert O.mp_constraint(2.0, u) == 2.0


def test_mp_ul_bound_sets_the_upper_limit():
    """Stencil (1.75, 1.875, 2, 5, 8): a gentle slope behind a jump.
    step 2: f* = 2 + minmod(3, 4 * 0.125) = 2.5: step 3 keeps (2, 2.5);
    step 4: d_{i-1} = 1.75 + 2 - 3.75 = 0, d_i = 1.875 + 5 - 4 = 2.875,
            d_{i+1} = 2 + 8 - 10 = 0; both d^M4 are 0 (a zero argument);
    step 5: f^UL = 2 + 0.5 = 2.5, f^MD = f^AV = 3.5, f^LC = 2.0625;
    step 6: f^min = max(min(2, 5, 3.5), min(2, 2.5, 2.0625)) = 2,
            f^max = min(max(2, 5, 3.5), max(2, 2.5, 2.0625)) = 2.5 (= f^UL).
    alpha = 2 would move f^max to 2.25."""
    u = _stencil5(1.75, 1.875, 2.0, 5.0, 8.0)
    assert O.mp_bounds(u) == (2.0, 2.5)
    assert O.mp_constraint(3.0, u) == 2.5
    assert O.mp_constraint(2.25, u) == 2.25
    assert O.mp_constraint(1.5, u) == 2.0
    assert O.mp_bounds(u, alpha=2.0) == (2.0, 2.25)


@pytest.mark.parametrize("order", [5, 7])
@pytest.mark.parametrize("n", [16, 32, 64, 128])
def test_mp_keeps_smooth_extrema(order, n):
    """Suresh & Huynh's design goal for steps 4-7: at a smooth extremum the
    constraint does not clip.  Exact cell averages of cos(2 pi x) on n cells:
    for every interface and CFL number the constrained CSL flux equals the
    unconstrained one.  Without the curvature terms of f^MD / f^LC the bounds
    at the peak collapse to the cell averages and clip the interpolant."""
    h = 1.0 / n
    a = np.arange(n) * h
    f = (np.sin(2 * np.pi * (a + h)) - np.sin(2 * np.pi * a)) / (2 * np.pi * h)
    for nu in (0.05, 0.2, 0.45):
        for i in range(n):
            u = np.array([f[(i + k) % n] for k in range(-3, 4)])
            phi = O.csl_flux(order, nu, u)
            assert O.mp_constraint(phi, u) == phi, (nu, i)


def test_pp_limiter_is_the_clamp_into_the_emptying_fluxes():
    """For f_i, f_{i+1} >= 0 and 0 < nu <= 1/2 the theta blend of Eqs. 15-23
    reduces to a clamp: when U+ < 0 it returns exactly the flux that empties
    the upwind cell, f_i / (2 nu) (theta+ (Phi - f_i) = (1 - 2 nu) f_i / (2 nu));
    when U- < 0 the flux that empties the downwind half, -f_{i+1} / (2 nu);
    both cannot bind at once.  So Phi^ = clamp(Phi, -f_{i+1}/(2 nu), f_i/(2 nu))
    up to the (1 - 8 eps) safety factor on theta."""
    rng = np.random.default_rng(31)
    for _ in range(3000):
        u0, u1 = rng.random(2) ** 3 * (rng.random(2) < 0.9)
        nu = float(rng.uniform(1e-3, 0.5))
        phi = float(rng.normal() * rng.choice([0.1, 1.0, 10.0]))
        want = min(max(phi, -u1 / (2 * nu)), u0 / (2 * nu))
        got = O.pp_limiter(phi, u0, u1, nu)
        assert abs(got - want) <= 2e-14 * max(abs(phi), u0 / nu, u1 / nu, 1e-300)


# ---- time step, Sec. 2.4 Eqs. 56-58 ----------------------------------------

def test_cfl_dt_hand_cases():
    """dt = min(dt_p, dt_v); dt_p = nu min_d (Delta x_d / V_d^max) with V_d^max
    the larger of |v_lo|, |v_hi|; dt_v = nu min over axes and mesh points of
    Delta v_d / |a_d|.  Binary-fraction grids so the expected values are exact.
    1D: Delta x = 0.0625 (16 cells on [0, 1]), v in [-2, 1] (V^max = 2),
        Delta v = 0.25 (12 cells): dt_p = 0.4 * 0.03125 = 0.0125;
        |a| <= 1: dt_v = 0.4 * 0.25 = 0.1 -> dt = 0.0125;
        |a| = 16 somewhere: dt_v = 0.4 * 0.015625 = 0.00625 -> dt = 0.00625.
    2D: Delta x = (0.0625, 0.25), V^max = (2, 4): dt_p = nu * min(0.03125, 0.0625);
        Delta v = (0.25, 0.25) with max |a| = (1, 16) on the two axes:
        dt_v = nu * 0.015625 (the second axis)."""
    g1 = O.grid(1, [16], [12], [0.0], [1.0], [-2.0], [1.0])
    assert O.cfl_dt(g1, 0.4) == pytest.approx(0.0125, rel=1e-15)
    assert O.cfl_dt(g1, 0.4, np.zeros(16)) == pytest.approx(0.0125, rel=1e-15)
    a = np.linspace(-1.0, 1.0, 16)
    assert O.cfl_dt(g1, 0.4, a) == pytest.approx(0.0125, rel=1e-15)
    a[5] = -16.0
    assert O.cfl_dt(g1, 0.4, a) == pytest.approx(0.00625, rel=1e-15)
    g2 = O.grid(2, [16, 8], [12, 18], [0.0, 0.0], [1.0, 2.0], [-2.0, -0.5], [1.0, 4.0])
    assert O.cfl_dt(g2, 0.2) == pytest.approx(0.2 * 0.03125, rel=1e-15)
    acc = np.zeros((2, g2.NX))
    acc[0, 3] = 1.0
    acc[1, 7] = -16.0
    assert O.cfl_dt(g2, 0.2, acc) == pytest.approx(0.2 * 0.015625, rel=1e-15)
    acc[1, 7] = 2.0   # dt_v = 0.2 * 0.125 > dt_p
    assert O.cfl_dt(g2, 0.2, acc) == pytest.approx(0.2 * 0.03125, rel=1e-15)

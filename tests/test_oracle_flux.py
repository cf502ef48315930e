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

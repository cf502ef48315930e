"""Pins of the oracle's Poisson solver and force (Sec. 2.2, Appendix C).

Pins: the closed-form potential and force of Appendix C with their orders
2/4/6; a dense linear solve of the same discrete Laplacian (brute force,
independent of any Fourier transform); direct summation of the isolated
Green function; numpy's FFT for the plain DFT; the potential of a Plummer
sphere.
"""
import math

import numpy as np
import pytest

import oracle as O


def _grid1d(n, L, order, coupling=4 * math.pi, rho_bg=0.0):
    return O.grid(1, [n], [2], [0.0], [L], [-1.0], [1.0], pois_order=order,
                  coupling=coupling, rho_bg=rho_bg)


def test_dft_matches_numpy_fft():
    rng = np.random.default_rng(0)
    for n in (1, 2, 7, 16, 33):
        x = rng.normal(size=n) + 1j * rng.normal(size=n)
        assert np.allclose(O.dft(x, -1), np.fft.fft(x), atol=1e-12 * n)
        assert np.allclose(O.dft(x, +1), np.fft.ifft(x) * n, atol=1e-12 * n)


@pytest.mark.parametrize("order", [2, 4, 6])
def test_appendix_c_convergence_orders(order):
    """rho = rho_bar (1 + A sin kx), k = 32 pi / L: phi and the force converge
    at the solver's order (Eqs. C12-C16, Fig. of Appendix C)."""
    L, rb, A, G = 1.0, 1.0, 0.5, 1.0
    k = 32 * math.pi / L
    ep, ef = [], []
    for n in (64, 128, 256, 512):
        g = _grid1d(n, L, order)
        x = g.x_centres(0)
        rho = rb * (1 + A * np.sin(k * x))
        phi, acc = O.poisson_solve(g, rho)
        phi_ex = -4 * math.pi * G * rb * A / k ** 2 * np.sin(k * x)
        f_ex = 4 * math.pi * G * rb * A / k * np.cos(k * x)
        ep.append(np.mean(np.abs(phi - phi_ex)))
        ef.append(np.mean(np.abs(acc[0] - f_ex)))
    sp = np.log2(np.array(ep[:-1]) / np.array(ep[1:]))
    sf = np.log2(np.array(ef[:-1]) / np.array(ef[1:]))
    # 4 points per wavelength at N = 64 is pre-asymptotic; the slopes approach
    # the order from below
    assert np.all(sp > order - 0.5) and sp[-1] > order - 0.1, (order, ep, sp)
    assert np.all(sf > order - 0.5) and sf[-1] > order - 0.1, (order, ef, sf)


def _stencil(order):
    if order == 2:
        return {0: -2.0, 1: 1.0, -1: 1.0}, 1.0
    if order == 4:
        return {0: -30.0, 1: 16.0, -1: 16.0, 2: -1.0, -2: -1.0}, 12.0
    return {0: -490.0, 1: 270.0, -1: 270.0, 2: -27.0, -2: -27.0, 3: 2.0, -3: 2.0}, 180.0


@pytest.mark.parametrize("order", [2, 4, 6])
def test_matches_dense_solve_of_discrete_laplacian_2d(order):
    """Brute force: build the periodic discrete Laplacian of Eqs. (C1, C5, C6)
    along each axis as a dense matrix, solve for the zero-mean potential and
    compare (no Fourier transform involved)."""
    nx, ny, Lx, Ly, S = 8, 6, 2.0, 1.5, -1.3
    g = O.grid(2, [nx, ny], [1, 1], [0, 0], [Lx, Ly], [-1, -1], [1, 1], pois_order=order,
               coupling=S, rho_bg=0.0)
    rng = np.random.default_rng(1)
    rho = rng.normal(size=nx * ny)
    phi, acc = O.poisson_solve(g, rho)
    st, den = _stencil(order)
    hx, hy = Lx / nx, Ly / ny
    n = nx * ny
    A = np.zeros((n, n))
    for i in range(nx):
        for j in range(ny):
            r = i * ny + j
            for o, c in st.items():
                A[r, ((i + o) % nx) * ny + j] += c / (den * hx * hx)
                A[r, i * ny + (j + o) % ny] += c / (den * hy * hy)
    b = S * (rho - rho.mean())
    sol = np.linalg.lstsq(A, b, rcond=None)[0]
    sol -= sol.mean()
    assert np.allclose(phi, sol, atol=1e-10 * np.abs(sol).max())


def test_force_is_minus_gradient_fda6():
    """accel = -(phi_{i+3} - 9 phi_{i+2} + 45 phi_{i+1} - 45 phi_{i-1} + ...)/60h
    evaluated independently from the returned phi."""
    n, L = 32, 3.0
    g = _grid1d(n, L, 6, coupling=-1.0, rho_bg=1.0)
    rho = 1 + 0.3 * np.cos(2 * math.pi * 3 * g.x_centres(0) / L) + 0.1 * np.sin(
        2 * math.pi * g.x_centres(0) / L)
    phi, acc = O.poisson_solve(g, rho)
    h = L / n
    r = lambda k: np.roll(phi, -k)
    want = -(r(3) - 9 * r(2) + 45 * r(1) - 45 * r(-1) + 9 * r(-2) - r(-3)) / (60 * h)
    assert np.allclose(acc[0], want, atol=1e-13)


def test_plasma_sign_convention():
    """Electrons (S = -1, rho_bg = 1): an excess of electrons pushes electrons
    away, i.e. the acceleration points down the density gradient."""
    n, L = 64, 4 * math.pi
    g = _grid1d(n, L, 6, coupling=-1.0, rho_bg=1.0)
    x = g.x_centres(0)
    rho = 1 + 0.1 * np.cos(0.5 * x)
    _, acc = O.poisson_solve(g, rho)
    # analytic: lap phi = -(rho - 1) -> phi = 0.1 cos(kx)/k^2; a = -phi' = 0.1 sin(kx)/k
    assert np.allclose(acc[0], 0.1 * np.sin(0.5 * x) / 0.5, rtol=1e-5, atol=1e-7)


def test_isolated_matches_direct_summation():
    """Doubling-up (Sec. 2.2) equals the direct sum of -(S/4pi) dV rho_j / r_ij
    with the cell-mean self term, on the box."""
    n, h, S = 5, 0.4, 4 * math.pi
    L = n * h
    g = O.grid(3, [n] * 3, [1] * 3, [0] * 3, [L] * 3, [-1] * 3, [1] * 3, poisson=O.POIS_ISOLATED,
               pois_order=6, coupling=S, rho_bg=0.0)
    rng = np.random.default_rng(2)
    rho = rng.random(n ** 3)
    phi, _ = O.poisson_solve(g, rho)
    idx = np.array(np.unravel_index(np.arange(n ** 3), (n, n, n))).T * h
    # mean of 1/r over a cube of side h about its centre, by quadrature: the
    # cube splits into 24 pyramids with apex at the centre, each giving
    # (h/2)^2 / 2 * I with I = int_0^1 int_0^1 (1 + u^2 + v^2)^(-1/2) du dv
    from scipy.integrate import dblquad
    I = dblquad(lambda v, u: (1 + u * u + v * v) ** -0.5, 0, 1, 0, 1, epsabs=1e-13)[0]
    self_mean = 3.0 * I / h
    want = np.zeros(n ** 3)
    for i in range(n ** 3):
        r = np.sqrt(((idx - idx[i]) ** 2).sum(axis=1))
        inv = np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), self_mean)
        want[i] = -(S / (4 * math.pi)) * h ** 3 * (rho * inv).sum()
    assert np.allclose(phi, want, rtol=1e-10, atol=0)


def test_isolated_plummer_potential():
    """Isolated solve of a Plummer density (G = M = a = 1) reproduces
    -GM / sqrt(r^2 + a^2) inside the box up to the mass outside the box and
    discretisation (a few percent)."""
    n, box = 16, 4.0
    g = O.grid(3, [n] * 3, [1] * 3, [-box] * 3, [box] * 3, [-1] * 3, [1] * 3,
               poisson=O.POIS_ISOLATED, pois_order=6, coupling=4 * math.pi, rho_bg=0.0)
    c = g.x_centres(0)
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    r2 = (X ** 2 + Y ** 2 + Z ** 2).ravel()
    rho = 3 / (4 * math.pi) * (1 + r2) ** -2.5
    phi, acc = O.poisson_solve(g, rho)
    ex = -1 / np.sqrt(r2 + 1)
    core = r2 < 4.0
    assert np.max(np.abs(phi[core] - ex[core]) / np.abs(ex[core])) < 0.08
    # radial force points inwards and has the right magnitude at r ~ 1
    a_r = (acc[0] * X.ravel() + acc[1] * Y.ravel() + acc[2] * Z.ravel()) / np.sqrt(r2)
    sel = (r2 > 0.5) & (r2 < 2.0)
    a_ex = -np.sqrt(r2[sel]) / (r2[sel] + 1) ** 1.5
    assert np.all(a_r[sel] < 0)
    assert np.max(np.abs(a_r[sel] - a_ex) / np.abs(a_ex)) < 0.1

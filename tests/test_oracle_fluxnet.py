"""Pins of the FP64 reference of the learned flux correction.

bfloat16 rounding against torch's own conversion; gradients against central
finite differences of the loss (independent of the backward code); simple
closed cases of the forward pass.
"""
import numpy as np
import pytest

from oracle import flux_net as N


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-8, 8, size=2000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 65504.0]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(N.bf16(x), want)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p = N.init_params(3)
    for k in p:  # move biases off zero so no ReLU sits exactly at its kink
        p[k] = p[k] + 0.05 * rng.normal(size=p[k].shape)
    X = rng.normal(size=(40, N.NFEAT))
    y = rng.normal(size=40)
    _, g = N.loss_and_grad(p, X, y, round_bf16=False)
    v = N.pack(p)
    gv = N.pack(g)
    eps = 1e-6
    idx = rng.choice(v.size, size=60, replace=False)
    for i in idx:
        vp, vm = v.copy(), v.copy()
        vp[i] += eps
        vm[i] -= eps
        lp, _ = N.loss_and_grad(N.unpack(vp), X, y, round_bf16=False)
        lm, _ = N.loss_and_grad(N.unpack(vm), X, y, round_bf16=False)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - gv[i]) <= 1e-6 * (1 + abs(fd)), (i, fd, gv[i])


def test_forward_closed_cases():
    p = {k: np.zeros(s) for k, s in N.SHAPES.items()}
    p["b4"] = np.array([0.375])
    X = np.random.default_rng(2).normal(size=(5, N.NFEAT))
    g, _ = N.forward(p, X)
    assert np.all(g == 0.375)
    # one active path: x_0 -> h1[0] -> h2[0] -> h3[0] -> g, all weights 1 (exact in bf16)
    p["W1"][0, 0] = p["W2"][0, 0] = p["W3"][0, 0] = p["w4"][0] = 1.0
    p["b4"] = np.array([0.0])
    X = np.zeros((3, N.NFEAT))
    X[:, 0] = [-1.0, 0.5, 2.0]
    g, _ = N.forward(p, X)
    assert np.array_equal(g, [0.0, 0.5, 2.0])


def test_features_are_scale_invariant():
    rng = np.random.default_rng(4)
    u, up, um = rng.random((10, 8)), rng.random((10, 8)), rng.random((10, 8))
    nu = rng.uniform(0, 0.5, 10)
    X1, s1 = N.features(u, up, um, nu)
    X2, s2 = N.features(1e-6 * u, 1e-6 * up, 1e-6 * um, nu)
    assert X1.shape == (10, N.NFEAT)
    assert np.allclose(X1, X2, rtol=1e-12, atol=1e-12)
    assert np.allclose(s2, 1e-6 * s1)
    assert np.all(X1[:, 3] == 0.0)
    assert np.array_equal(X1[:, 24], nu)


def test_features_velocity_difference_and_curvature():
    # a line between neighbours that differ by a constant c has velocity
    # difference features c / (2 s) everywhere; equal neighbours give zero
    u = np.full((1, 8), 2.0)
    X, s = N.features(u, u + 0.5, u - 0.5, np.array([0.25]))
    assert np.allclose(X[0, 8:16], 0.5 / 2.0)
    assert np.allclose(X[0, 16:24], 0.0)
    X, _ = N.features(u, u, u, np.array([0.25]))
    assert np.all(X[0, 8:24] == 0.0)
    # a parabola in v: neighbours both 1 above gives curvature 2 / (2 s)
    X, _ = N.features(u, u + 1.0, u + 1.0, np.array([0.25]))
    assert np.allclose(X[0, 8:16], 0.0) and np.allclose(X[0, 16:24], 1.0 / 2.0)


def test_pair_loss_gradients_match_finite_differences():
    # the cell-update loss: groups of two with coefficients a_k
    rng = np.random.default_rng(5)
    p = N.init_params(6)
    for k in p:
        p[k] = p[k] + 0.05 * rng.normal(size=p[k].shape)
    X = rng.normal(size=(30, N.NFEAT))
    y = rng.normal(size=30)
    a = rng.uniform(-1, 1, size=30)
    loss, g = N.loss_and_grad(p, X, y, round_bf16=False, coef=a, group=2)
    gx, _ = N.forward(p, X, round_bf16=False)
    r = (a * (gx - y)).reshape(-1, 2).sum(axis=1)
    assert loss == pytest.approx(float(np.mean(r * r)), rel=1e-12)
    v, gv = N.pack(p), N.pack(g)
    eps = 1e-6
    for i in rng.choice(v.size, size=40, replace=False):
        vp, vm = v.copy(), v.copy()
        vp[i] += eps
        vm[i] -= eps
        lp, _ = N.loss_and_grad(N.unpack(vp), X, y, round_bf16=False, coef=a, group=2)
        lm, _ = N.loss_and_grad(N.unpack(vm), X, y, round_bf16=False, coef=a, group=2)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - gv[i]) <= 1e-6 * (1 + abs(fd)), (i, fd, gv[i])


# ---- the learned line update (oracle/flux_net.learned_line) -----------------
#
# Pinned by properties that hold whatever the network: the flux form conserves
# mass on a periodic line, the mass-form PP limiter keeps f >= 0, an integer
# shift moves no mass through any interface, a zero network reduces to the
# plain SL-MPP7 update of the oracle, and the MP bounds remove a correction
# on data where they have zero width.

import oracle as O  # noqa: E402


def _rand_params(seed, scale):
    p = N.init_params(seed)
    rng = np.random.default_rng(seed + 7)
    for k in p:
        p[k] = p[k] * scale + 0.05 * scale * rng.normal(size=p[k].shape)
    return p


def _lines(rng, L, zeros=0.3):
    f = rng.random(L) ** rng.choice([1, 3, 6]) * (rng.random(L) >= zeros)
    up = rng.random(L) * (rng.random(L) >= zeros)
    um = rng.random(L) * (rng.random(L) >= zeros)
    return f, up, um


@pytest.mark.parametrize("mpb", [False, True])
def test_learned_line_with_zero_network_is_the_plain_update(mpb):
    rng = np.random.default_rng(40)
    p = {k: np.zeros(s) for k, s in N.SHAPES.items()}
    for _ in range(60):
        L = int(rng.integers(8, 30))
        f, up, um = _lines(rng, L)
        s = float(rng.uniform(-4, 4))
        bc = int(rng.integers(0, 2))
        got = N.learned_line(f, up, um, s, p, bc, mp_bound=mpb)
        want = O.advect_line(f, s, order=7, mp=1, pp=1, bc=bc)
        assert np.abs(got - want).max() <= 1e-15 * max(f.max(), 1e-300), s


@pytest.mark.parametrize("mpb", [False, True])
def test_learned_line_conserves_mass_and_positivity_for_any_network(mpb):
    rng = np.random.default_rng(41)
    for t in range(60):
        p = _rand_params(t, scale=float(rng.choice([1.0, 5.0, 30.0])))
        L = int(rng.integers(8, 30))
        f, up, um = _lines(rng, L)
        s = float(rng.uniform(-3, 3))
        got = N.learned_line(f, up, um, s, p, O.BC_PERIODIC, mp_bound=mpb)
        assert got.min() >= 0.0
        assert abs(got.sum() - f.sum()) <= 1e-14 * max(f.sum(), 1e-300)
        out = N.learned_line(f, up, um, s, p, O.BC_OUTFLOW, mp_bound=mpb)
        assert out.min() >= 0.0


def test_learned_line_integer_shift_is_exact_with_mp_bounds():
    """nu = 0 with the MP bounds on: in mass form they have zero width, so the
    network can move nothing and the line is shifted cell for cell."""
    rng = np.random.default_rng(42)
    p = _rand_params(3, scale=10.0)
    for n in (-5, -1, 0, 2, 7):
        f, up, um = _lines(rng, 19)
        got = N.learned_line(f, up, um, float(n), p, O.BC_PERIODIC, mp_bound=True)
        assert np.array_equal(got, np.roll(f, n))
        out = N.learned_line(f, up, um, float(n), p, O.BC_OUTFLOW, mp_bound=True)
        want = np.zeros(19)
        if n >= 0:
            want[n:] = f[:19 - n]
        else:
            want[:n] = f[-n:]
        assert np.array_equal(out, want)


def test_learned_line_correction_obeys_the_mp_bounds():
    """On a constant line every MP bound is the constant itself, so with the
    bounds on any network's correction is cut back to nu f and the line does
    not change; without them a network whose output varies between
    interfaces (random velocity-neighbour lines) moves mass.  On a rising
    linear ramp (zero-inflow ends far from the cells checked) the bounds are
    [f_i, f_{i+1}] and a small constant g passes in both modes: each interior
    cell changes by -(s_out - s_in) g relative to the plain update, s = max |u|
    over the interface's 8-cell stencil."""
    rng = np.random.default_rng(43)
    p = _rand_params(5, scale=3.0)
    f = np.full(16, 0.5)
    up, um = rng.random(16), rng.random(16)
    for s in (0.3, -0.3, 2.4):
        assert np.array_equal(N.learned_line(f, up, um, s, p, O.BC_PERIODIC, mp_bound=True), f)
        assert not np.array_equal(N.learned_line(f, up, um, s, p, O.BC_PERIODIC), f)
    p = {k: np.zeros(s) for k, s in N.SHAPES.items()}
    z = np.zeros(40)
    ramp = 1.0 + 0.125 * np.arange(40)
    g = 1e-4
    p["b4"] = np.array([g])
    nu = 0.25
    plain = O.advect_line(ramp, nu, order=7, mp=1, pp=1, bc=O.BC_OUTFLOW)
    for mpb in (False, True):
        got = N.learned_line(ramp, z, z, nu, p, O.BC_OUTFLOW, mp_bound=mpb)
        # flow to the right: the interface right of cell i has stencil cells
        # i-3 .. i+4, so s_out = ramp[i+4] and s_in = ramp[i+3]
        for i in range(10, 30):
            assert got[i] - plain[i] == pytest.approx(-(ramp[i + 4] - ramp[i + 3]) * g, rel=1e-9, abs=1e-17)

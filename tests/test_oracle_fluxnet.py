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

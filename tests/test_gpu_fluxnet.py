"""Learned flux correction: training kernels against the FP64 reference,
the learned spatial sweep against the plain sweep and an oracle line update
(with the velocity-neighbour features),
conservation and positivity with the network on, the fine-flux extraction
used to build training data, and what a trained network gains."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import flux_net as N
from paper_1702_08521_gb300 import inputs
from paper_1702_08521_gb300 import vlasov as V

from gpu_helpers import both, from_gpu, rel_l1, rel_max, snapshot, to_gpu

pytestmark = pytest.mark.gpu


def _t(a, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _params(seed, scale=1.0):
    p = N.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    for k in p:
        p[k] = _f32(p[k] * scale + 0.02 * rng.normal(size=p[k].shape))
    return p


def test_net_gradients_match_reference():
    import torch
    rng = np.random.default_rng(0)
    p = _params(1)
    B = 1000
    X = _f32(rng.normal(size=(B, N.NFEAT)))
    y = _f32(rng.normal(size=B))
    loss_ref, g_ref = N.loss_and_grad(p, X, y, round_bf16=True)
    w = _t(N.pack(p), torch.float32)
    grad = torch.zeros_like(w)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    V.vp_net_grad(_t(X.ravel(), torch.float32), _t(y, torch.float32), B, w, grad, loss)
    torch.cuda.synchronize()
    assert loss.item() == pytest.approx(loss_ref, rel=1e-4)
    gv = grad.double().cpu().numpy()
    rv = N.pack(g_ref)
    assert np.abs(gv - rv).max() <= 1e-2 * np.abs(rv).max()
    assert np.linalg.norm(gv - rv) <= 1e-3 * np.linalg.norm(rv)


def test_pair_loss_gradients_match_reference():
    import torch
    rng = np.random.default_rng(2)
    p = _params(3)
    B = 1000
    X = _f32(rng.normal(size=(B, N.NFEAT)))
    y = _f32(rng.normal(size=B))
    a = _f32(rng.uniform(-1, 1, size=B))
    loss_ref, g_ref = N.loss_and_grad(p, X, y, round_bf16=True, coef=a, group=2)
    w = _t(N.pack(p), torch.float32)
    grad = torch.zeros_like(w)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    V.vp_net_grad(_t(X.ravel(), torch.float32), _t(y, torch.float32), B, w, grad, loss,
                  coef=_t(a, torch.float32), group=2)
    torch.cuda.synchronize()
    assert loss.item() == pytest.approx(loss_ref, rel=1e-4)
    gv = grad.double().cpu().numpy()
    rv = N.pack(g_ref)
    assert np.abs(gv - rv).max() <= 1e-2 * np.abs(rv).max()
    assert np.linalg.norm(gv - rv) <= 1e-3 * np.linalg.norm(rv)


def test_adam_moves_against_the_gradient():
    import torch
    w = torch.zeros(V.VP_NET_NPARAM, dtype=torch.float32, device="cuda")
    g = torch.linspace(-1, 1, V.VP_NET_NPARAM, device="cuda")
    m, v = torch.zeros_like(w), torch.zeros_like(w)
    g0 = g.clone()
    V.vp_net_adam(w, m, v, g, 1, 1e-3)
    torch.cuda.synchronize()
    # first Adam step moves every parameter by -lr * g / (|g| + eps), i.e.
    # -lr * sign(g) wherever |g| >> eps
    nz = g0.abs() > 1e-4
    assert torch.allclose(w[nz], -1e-3 * torch.sign(g0[nz]), rtol=1e-3, atol=1e-7)
    assert torch.count_nonzero(g) == 0


def _grid2d(nx, nv):
    L = 4 * math.pi
    return dict(dims=2, nx=[nx, nx], nv=[nv, nv], xlo=[0.0, 0.0], xhi=[L, L], vlo=[-6.0, -6.0],
                vhi=[6.0, 6.0], order=7)


def test_learned_sweep_without_net_is_the_plain_sweep():
    import torch
    g = _grid2d(8, 16)
    sim, og = both(g, V.VP_F32)
    f0 = inputs.random_f(og.NX * og.NV, seed=3).astype(np.float32)
    acc = inputs.random_accel(og.NX, 2, seed=4, amax=3.0)
    w = torch.zeros(V.VP_NET_NPARAM, dtype=torch.float32, device="cuda")
    for kick in (0, 1):
        for d in range(2):
            to_gpu(sim, f0)
            a = _t(acc[d])
            if kick:
                V.vp_kick_sweep(sim.ctx, d, 0.4, a)
            else:
                V.vp_drift_sweep(sim.ctx, d, 0.4)
            ref = from_gpu(sim)
            to_gpu(sim, f0)
            V.vp_learned_sweep(sim.ctx, kick, d, 0.4, a, w, 0)
            got = from_gpu(sim)
            assert rel_max(got, ref) <= 1e-6, (kick, d)
    sim.close()


@pytest.mark.parametrize("use_net", [1, 2])
def test_learned_sweep_matches_oracle_line_update(use_net):
    """use_net 1: PP on the corrected mass; 2: the MP bounds of App. A on it
    first (the oracle's mp_bound)."""
    import torch
    g = dict(dims=1, nx=[24], nv=[20], xlo=[0.0], xhi=[2.0], vlo=[-3.0], vhi=[3.0], order=7)
    sim, og = both(g, V.VP_F32)
    f0 = _f32(inputs.random_f(og.NX * og.NV, seed=5))
    p = _params(7, scale=0.3)
    w = _t(N.pack(p), torch.float32)
    to_gpu(sim, f0)
    V.vp_learned_sweep(sim.ctx, 0, 0, 0.37, None, w, use_net, snapshot(sim))
    got = from_gpu(sim).reshape(24, 20)
    want = np.empty((24, 20))
    f2 = f0.reshape(24, 20)
    vc = og.v_centres(0)
    zero = np.zeros(24)
    for j in range(20):
        s = vc[j] * 0.37 / (2.0 / 24)
        sp = 1 if vc[j] >= 0 else -1
        up = f2[:, j + sp] if 0 <= j + sp < 20 else zero
        um = f2[:, j - sp] if 0 <= j - sp < 20 else zero
        want[:, j] = N.learned_line(f2[:, j], up, um, s, p, O.BC_PERIODIC, mp_bound=use_net == 2)
    # FP32 sums vs FP64 sums can move a bfloat16 rounding by one step
    assert rel_l1(got, want) <= 2e-3, rel_l1(got, want)
    sim.close()


def test_learned_sweep_integer_shift_is_exact_with_mp_bounds():
    """An integer shift (nu = 0 on every line) with the network on and the MP
    bounds applied to its correction (use_net = 2): in mass form they have
    zero width, so the learned sweep is the exact shift of every line, bit
    for bit, as in the oracle's learned update."""
    import torch
    g = dict(dims=1, nx=[24], nv=[20], xlo=[0.0], xhi=[24.0], vlo=[-5.0], vhi=[5.0], order=7)
    sim, og = both(g, V.VP_F32)
    f0 = _f32(inputs.random_f(og.NX * og.NV, seed=15))
    w = _t(N.pack(_params(9, scale=3.0)), torch.float32)
    to_gpu(sim, f0)
    # dx = 1, v_j = -4.75 + 0.5 j, dt = 4: shift v_j dt = -19 + 2 j cells
    dt = 4.0
    V.vp_learned_sweep(sim.ctx, 0, 0, dt, None, w, 2, snapshot(sim))
    got = from_gpu(sim).reshape(24, 20)
    f2 = f0.reshape(24, 20)
    for j, v in enumerate(og.v_centres(0)):
        n = int(round(v * dt))
        assert v * dt == n
        assert np.array_equal(got[:, j], np.roll(f2[:, j], n)), j
    sim.close()


def test_learned_sweep_conserves_mass_and_positivity():
    import torch
    g = _grid2d(8, 16)
    sim, og = both(g, V.VP_F32)
    f0 = (inputs.random_f(og.NX * og.NV, seed=9, zeros=0.4) ** 4).astype(np.float32)
    p = _params(11, scale=3.0)  # a large, untrained correction
    w = _t(N.pack(p), torch.float32)
    to_gpu(sim, f0)
    m0 = float(np.sum(f0, dtype=np.float64))
    for _ in range(3):
        for d in range(2):
            V.vp_learned_sweep(sim.ctx, 0, d, 0.3, None, w, 1, snapshot(sim))
    got = from_gpu(sim)
    assert got.min() >= 0.0
    assert abs(got.sum() - m0) / m0 <= 1e-6
    sim.close()


def test_fine_flux_reproduces_the_sweep():
    import torch
    g = _grid2d(8, 16)
    sim, og = both(g, V.VP_F32)
    f0 = inputs.random_f(og.NX * og.NV, seed=12).astype(np.float32)
    acc = inputs.random_accel(og.NX, 2, seed=13, amax=8.0)
    for kick, d in ((0, 0), (0, 1), (1, 0), (1, 1)):
        to_gpu(sim, f0)
        a = _t(acc[d])
        L = g["nv"][d] if kick else g["nx"][d]
        nlines = og.NX * og.NV // L
        G = torch.zeros(nlines * (L + 1), dtype=torch.float64, device="cuda")
        V.vp_fine_flux(sim.ctx, kick, d, 0.55, a, 1, G)
        if kick:
            V.vp_kick_sweep(sim.ctx, d, 0.55, a)
        else:
            V.vp_drift_sweep(sim.ctx, d, 0.55)
        ref = from_gpu(sim)
        Gh = G.cpu().numpy().reshape(nlines, L + 1)
        # rebuild f' = f + G_{i-1/2} - G_{i+1/2} along every line
        shp = og.shape
        axis = (2 + d) if kick else d
        fl = np.moveaxis(f0.reshape(shp).astype(np.float64), axis, -1)
        lines = fl.reshape(-1, L)
        order = np.arange(np.prod(shp)).reshape(shp)
        idx = np.moveaxis(order, axis, -1).reshape(-1, L)
        # G rows follow the library's line order: [outer][inner]
        outer = int(np.prod(shp[:axis]))
        inner = int(np.prod(shp[axis + 1:]))
        lib_first = (np.arange(outer)[:, None] * L * inner + np.arange(inner)[None, :]).ravel()
        pos = {v: k for k, v in enumerate(idx[:, 0])}
        rows = np.array([pos[v] for v in lib_first])
        new = lines[rows] + Gh[:, :-1] - Gh[:, 1:]
        got = np.empty(np.prod(shp))
        got[idx[rows].ravel()] = new.ravel()
        assert rel_max(got, ref) <= 1e-5, (kick, d, rel_max(got, ref))
    sim.close()


def test_learned_correction_rejects_velocity_sweeps():
    import torch
    g = _grid2d(8, 16)
    sim, og = both(g, V.VP_F32)
    w = torch.zeros(V.VP_NET_NPARAM, dtype=torch.float32, device="cuda")
    acc = _t(inputs.random_accel(og.NX, 2, seed=4, amax=3.0)[0])
    with pytest.raises(V.VpError):
        V.vp_learned_sweep(sim.ctx, 1, 0, 0.4, acc, w, 1, snapshot(sim))
    sim.close()


def test_learned_step_replays_the_sweep_sequence():
    """vp_learned_step (captured in a CUDA graph) gives, bit for bit, the f
    of the same KDK sequence issued sweep by sweep: plain kicks, learned
    drifts (library snapshot), field solve between; and a plain vp_step
    is unchanged by the learned path having run on the context."""
    import torch
    g = _grid2d(8, 16)
    f0 = (inputs.random_f(8 * 8 * 16 * 16, seed=21, zeros=0.3) ** 2).astype(np.float32)
    w = _t(N.pack(_params(5, scale=0.5)), torch.float32)
    dt = 0.2
    a, _ = both(g, V.VP_F32)
    b, _ = both(g, V.VP_F32)
    for sim in (a, b):
        to_gpu(sim, f0)
        sim.field()
    a.learned_step(dt, 3, w)
    a.sync()
    for _ in range(3):
        for d in range(2):
            V.vp_kick_sweep(b.ctx, d, 0.5 * dt, b.accel[d * b.NX:])
        for d in (1, 0):
            V.vp_learned_sweep(b.ctx, 0, d, dt, None, w, 1)
        b.field()
        for d in range(2):
            V.vp_kick_sweep(b.ctx, d, 0.5 * dt, b.accel[d * b.NX:])
    b.sync()
    fa, fb = from_gpu(a), from_gpu(b)
    assert np.array_equal(fa, fb)
    assert fa.min() >= 0.0
    # the plain step on the same contexts still matches sweep by sweep
    a.step(dt, 1)
    a.sync()
    for d in range(2):
        V.vp_kick_sweep(b.ctx, d, 0.5 * dt, b.accel[d * b.NX:])
    for d in (1, 0):
        V.vp_drift_sweep(b.ctx, d, dt)
    b.field()
    for d in range(2):
        V.vp_kick_sweep(b.ctx, d, 0.5 * dt, b.accel[d * b.NX:])
    b.sync()
    assert np.array_equal(from_gpu(a), from_gpu(b))
    a.close()
    b.close()


def test_learned_sweep_velocity_axis_limit():
    """One 128-row MMA operand per interface step: 128 velocity cells on the
    sweep's velocity axis run (mass kept, f >= 0), 129 are refused with
    VP_ENOTSUP and f is left as it was."""
    import torch
    w = _t(N.pack(_params(5, 0.3)), torch.float32)
    for nv, ok in ((128, True), (129, False)):
        g = dict(dims=1, nx=[16], nv=[nv], xlo=[0.0], xhi=[4.0], vlo=[-3.0], vhi=[3.0], order=7)
        sim, og = both(g, V.VP_F32)
        f0 = _f32(inputs.random_f(og.NX * og.NV, seed=nv))
        to_gpu(sim, f0)
        if ok:
            V.vp_learned_sweep(sim.ctx, 0, 0, 0.3, None, w, 1)
            f1 = from_gpu(sim)
            assert f1.min() >= 0.0
            assert abs(f1.sum() - f0.sum()) <= 1e-5 * f0.sum()
        else:
            with pytest.raises(V.VpError) as e:
                V.vp_learned_sweep(sim.ctx, 0, 0, 0.3, None, w, 1)
            assert e.value.code == V.VP_ENOTSUP
            assert np.array_equal(from_gpu(sim), f0)
        sim.close()

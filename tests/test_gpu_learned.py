"""What a trained flux-correction network gains over the plain coarse scheme.

A small 2D2V Landau setup: pairs from fine-grid (16^2 x 64^2) runs of the
method, a network trained on the GPU, then on a held-out state (k = 0.5,
alpha = 0.05, after 8 fine steps) every spatial sweep of one step is done
three ways on the 16^2 x 16^2 grid: plain MP7, learned, and the restricted
fine sweep (the target).  The learned sweeps must land closer to the target
than the plain ones.  A 20-step run of both against the fine FP64 oracle
must not be worse with the network; its gain is printed.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1702_08521_gb300 import learned as LR
from paper_1702_08521_gb300 import vlasov as V

pytestmark = pytest.mark.gpu

DIMS, NX, NVF, FACTOR, DT = 2, 16, 64, 4, 0.1


@pytest.fixture(scope="module")
def trained():
    import torch
    stream = torch.cuda.Stream()
    rng = np.random.Generator(np.random.PCG64(1703))
    Xs, ys, cs = [], [], []
    for _ in range(6):
        k = float(rng.uniform(0.3, 0.6))
        a = float(rng.uniform(0.01, 0.1))
        S = LR.Sampler(DIMS, NX, NVF, FACTOR, k, stream)
        X, y, c = S.run_draw(k, a, DT, steps=12, every_step=2, zmin=0.0, keep=20000, rng=rng, importance=2.0)
        Xs += X
        ys += y
        cs += c
        S.close()
    X = torch.cat(Xs)
    y = torch.cat(ys)
    c = torch.cat(cs)
    w, hist = LR.train_net(X, y, iters=1500, batch=16384, lr=2e-3, stream=stream, coef=c)
    torch.cuda.synchronize()
    r0 = float(((c * y).view(-1, 2).sum(dim=1) ** 2).mean())  # the loss of g = 0
    assert hist[-1] < r0  # the fit explains part of the cell-update error
    return w, stream


def _rel(a, b):
    a, b = a.double(), b.double()
    return float((a - b).abs().sum() / b.abs().sum())


def test_learned_velocity_sweeps_are_closer_to_the_fine_target(trained):
    import torch
    w, stream = trained
    S = LR.Sampler(DIMS, NX, NVF, FACTOR, 0.5, stream)
    V.vp_init_f(S.fine.ctx, *LR._landau_ic(DIMS, 0.5, 0.05))
    S.fine.field()
    for _ in range(8):
        for sw in LR._sweeps(DIMS):
            if sw is None:
                S.fine.field()
                continue
            kick, d, fac = sw
            acc = S.fine.accel[d * S.fine.NX:] if kick else None
            if kick:
                V.vp_kick_sweep(S.fine.ctx, d, fac * DT, acc)
            else:
                V.vp_drift_sweep(S.fine.ctx, d, fac * DT)
    gains = []
    stream.synchronize()
    for d in (1, 0):  # x2 then x1, as in the step
        S.restrict()
        stream.synchronize()
        f0 = S.coarse.f.clone()
        torch.cuda.synchronize()
        V.vp_drift_sweep(S.coarse.ctx, d, DT)
        stream.synchronize()
        plain = S.coarse.f.clone()
        S.coarse.f.copy_(f0)
        torch.cuda.synchronize()
        V.vp_learned_sweep(S.coarse.ctx, 0, d, DT, None, w, 1, f0)
        stream.synchronize()
        learned = S.coarse.f.clone()
        # the same sweep with the MP bounds of App. A on the corrected mass
        S.coarse.f.copy_(f0)
        torch.cuda.synchronize()
        V.vp_learned_sweep(S.coarse.ctx, 0, d, DT, None, w, 2, f0)
        stream.synchronize()
        learned_mp = S.coarse.f.clone()
        S.coarse.f.copy_(learned)
        torch.cuda.synchronize()
        V.vp_drift_sweep(S.fine.ctx, d, DT)
        S.restrict()
        stream.synchronize()
        target = S.coarse.f.clone()
        torch.cuda.synchronize()
        # error of the update itself, relative to the update's size
        upd = (target.double() - f0.double()).abs().sum()
        e_plain = float((plain.double() - target.double()).abs().sum() / upd)
        e_learn = float((learned.double() - target.double()).abs().sum() / upd)
        e_mp = float((learned_mp.double() - target.double()).abs().sum() / upd)
        print(f"spatial sweep x{d + 1}: plain {e_plain:.3e}, learned {e_learn:.3e}, "
              f"learned with MP bounds {e_mp:.3e} (of the update)")
        gains.append((e_plain, e_learn))
    S.close()
    for e_plain, e_learn in gains:
        assert e_learn < e_plain


def test_learned_run_against_fine_oracle_is_reported(trained):
    import torch
    w, stream = trained
    steps, k, a = 20, 0.5, 0.05
    f_fine = LR.restricted_initial_state(DIMS, NX, NVF, 1, k, a, stream)
    fc0 = LR.restricted_initial_state(DIMS, NX, NVF, FACTOR, k, a, stream)
    gc = LR.landau_grid(DIMS, NX, NVF // FACTOR, k)
    plain = LR.run(gc, fc0, DT, steps, None, stream)
    learned = LR.run(gc, fc0, DT, steps, w, stream)
    # fine FP64 oracle from the same (FP32-rounded) fine state
    og = O.grid(**LR.landau_grid(DIMS, NX, NVF, k))
    f = f_fine.double().cpu().numpy()
    _, _, acc = O.field(og, f)
    O.step(og, f, DT, steps, np.ascontiguousarray(acc), split=O.SPLIT_KDK)
    ref = f.reshape(NX * NX, NVF // FACTOR, FACTOR, NVF // FACTOR, FACTOR).mean(axis=(2, 4)).ravel()
    ref_t = torch.as_tensor(ref, device="cuda")
    e_p = _rel(plain.f, ref_t)
    e_l = _rel(learned.f, ref_t)
    print(f"20-step L1 vs fine FP64 oracle: plain {e_p:.4e}, learned {e_l:.4e}, gain {e_p / e_l:.3f}x")
    for sim in (plain, learned):
        assert float(sim.f.min()) >= 0.0
    m0 = float(fc0.double().sum())
    assert abs(float(learned.f.double().sum()) - m0) / m0 < 1e-5
    assert math.isfinite(e_l) and e_l < e_p
    plain.close()
    learned.close()


def test_fine_reference_of_the_learned_benchmark_matches_oracle():
    """The learned benchmark judges its runs against the GPU's FP64 run of the
    fine 2D2V Landau grid (k = 0.5, alpha = 0.05, KDK, dt = 0.1, t = 2).  That
    reference path, at a reduced 32^2 x 64^2 grid over the same 20 steps,
    equals the FP64 oracle from the same initial state."""
    import torch
    stream = torch.cuda.Stream()
    nx, nv, k, a = 32, 64, 0.5, 0.05
    f0 = LR.restricted_initial_state(2, nx, nv, 1, k, a, stream).double()
    g = LR.landau_grid(2, nx, nv, k)
    ref = LR.run(g, f0, DT, 20, None, stream, V.VP_F64)
    og = O.grid(**g)
    f = f0.cpu().numpy().copy()
    _, _, acc = O.field(og, f)
    O.step(og, f, DT, 20, np.ascontiguousarray(acc), split=O.SPLIT_KDK)
    got = ref.f.double().cpu().numpy()
    assert float(np.abs(got - f).max() / np.abs(f).max()) <= 1e-11
    ref.close()

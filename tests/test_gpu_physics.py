"""Physical checks of the whole path around the sweeps.

The self-gravitating Plummer sphere, 16^3 x 32^3 FP32: the sampled
distribution function starts near virial equilibrium (the oracle's FP64 value
of (2K + W) / |W| for this truncated box and grid is 0.022), and over 10 DKD
steps (t = 0.5) the equilibrium stays put: mass, virial ratio and the density
profile change only by the discretisation's drift.

The self-gravitating slab of Sec. 3.2 (periodic gravity in 1D1V): the FP64
run equals the oracle, and the FP32 run's mode grows (k/k_J = 0.5) or decays
(1.1) at the root of the kinetic dispersion relation."""
import numpy as np
import pytest

import oracle as O
from paper_1702_08521_gb300 import inputs
from paper_1702_08521_gb300 import vlasov as V

from gpu_helpers import both, from_gpu, rel_max, to_gpu
from test_oracle_vp import jeans_growth_root, jeans_least_damped_root

pytestmark = pytest.mark.gpu


def test_plummer_stays_near_equilibrium():
    cfg = inputs.plummer(16, 32)
    sim = V.Simulation(cfg["grid"], precision=V.VP_F32)
    V.vp_init_f(sim.ctx, *cfg["ic"])
    sim.field()
    d0 = sim.diagnostics()
    og = O.grid(**cfg["grid"])
    do = O.diagnostics(og, O.init_f(og, *cfg["ic"]))
    for k in ("mass", "ke", "pe"):
        assert d0[k] == pytest.approx(do[k], rel=1e-5), k
    vir0 = (2 * d0["ke"] + d0["pe"]) / abs(d0["pe"])
    assert abs(vir0) < 0.03, vir0
    rho0 = sim.rho.double().cpu().numpy().copy()
    sim.step(cfg["dt"], 10, split=cfg["split"])
    sim.field()
    d1 = sim.diagnostics()
    rho1 = sim.rho.double().cpu().numpy()
    vir1 = (2 * d1["ke"] + d1["pe"]) / abs(d1["pe"])
    dm = abs(d1["mass"] - d0["mass"]) / d0["mass"]
    drho = float(np.abs(rho1 - rho0).sum() / np.abs(rho0).sum())
    print(f"virial {vir0:.4f} -> {vir1:.4f}, mass change {dm:.2e}, density L1 change {drho:.3e}")
    assert d1["min_f"] >= 0.0
    assert dm < 1e-2
    assert abs(vir1) < 0.05
    assert drho < 0.05
    sim.close()


def _slab_run(ratio, precision, dt, steps):
    import torch
    cfg = inputs.jeans_slab(ratio, 64, amp=1e-3, precision="f64" if precision == V.VP_F64 else "f32")
    sim, og = both(cfg["grid"], precision)
    f_o = O.init_f(og, *cfg["ic"])
    if precision == V.VP_F32:
        f_o = f_o.astype(np.float32).astype(np.float64)
    to_gpu(sim, f_o)
    sim.field()
    d_dev = torch.zeros(steps * V.VP_NDIAG, dtype=torch.float64, device="cuda")
    sim.step(dt, steps, split=cfg["split"], mode=cfg["mode"], diag=d_dev)
    f_g = from_gpu(sim)
    d_g = d_dev.cpu().numpy().reshape(steps, V.VP_NDIAG)
    sim.close()
    return cfg, og, f_o, f_g, d_g


@pytest.mark.parametrize("ratio,t0,t1", [(0.5, 0.8, 1.6), (1.1, 1.0, 3.0)])
def test_self_gravitating_slab(ratio, t0, t1):
    """64 x 64, A = 1e-3, dt = 0.005 to t1: FP64 GPU against the oracle (f
    within 1e-12 relative max, |a_k| history within 1e-10); the slope of
    ln|a_k| of the FP32 GPU run over [t0, t1] within 0.5% of the growing
    (k/k_J = 0.5) or least damped (1.1) root."""
    dt = 0.005
    steps = int(round(t1 / dt))
    cfg, og, f_o, f_g, d_g = _slab_run(ratio, V.VP_F64, dt, steps)
    _, _, acc = O.field(og, f_o)
    acc = np.ascontiguousarray(acc)
    d_o = O.step(og, f_o, dt, steps, acc, split=cfg["split"], mode=cfg["mode"], diag=True)
    assert rel_max(f_g, f_o) <= 1e-12
    assert np.abs(d_g[:, 6] - d_o[:, 6]).max() <= 1e-10 * np.abs(d_o[:, 6]).max()
    _, _, _, f32, d32 = _slab_run(ratio, V.VP_F32, dt, steps)
    t = dt * np.arange(1, steps + 1)
    sel = (t >= t0 - 1e-9) & (t <= t1 + 1e-9)
    rate = np.polyfit(t[sel], np.log(d32[sel, 6]), 1)[0]
    want = jeans_growth_root(ratio) if ratio < 1 else jeans_least_damped_root(ratio).imag
    assert rate == pytest.approx(want, rel=5e-3), (rate, want)
    assert f32.min() >= 0.0


def test_uniform_sphere_ic_and_steps_match_oracle():
    """Sec. 3.4 sphere at 16^3 x 8^3 (FP64): the initial state equals the
    oracle's, and so does the state after 3 DKD steps of dt = 0.05."""
    cfg = inputs.uniform_sphere(16, 8, precision="f64")
    sim, og = both(cfg["grid"], V.VP_F64)
    V.vp_init_f(sim.ctx, *cfg["ic"])
    f_o = O.init_f(og, *cfg["ic"])
    assert rel_max(from_gpu(sim), f_o) <= 1e-14
    sim.field()
    _, _, acc = O.field(og, f_o)
    acc = np.ascontiguousarray(acc)
    sim.step(0.05, 3, split=cfg["split"])
    O.step(og, f_o, 0.05, 3, acc, split=cfg["split"], mode=1)
    assert rel_max(from_gpu(sim), f_o) <= 1e-12
    sim.close()

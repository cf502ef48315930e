"""Physical checks of the whole 3D3V path (a7-a10 around the sweeps) on the
self-gravitating Plummer sphere, 16^3 x 32^3 FP32: the sampled distribution
function starts near virial equilibrium (the oracle's FP64 value of
(2K + W) / |W| for this truncated box and grid is 0.022), and over 10 DKD
steps (t = 0.5) the equilibrium stays put: mass, virial ratio and the
density profile change only by the discretisation's drift."""
import numpy as np
import pytest

import oracle as O
from paper_1702_08521_gb300 import inputs
from paper_1702_08521_gb300 import vlasov as V

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

"""GPU parity of whole Strang-split runs against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1702_08521_gb300 import inputs
from paper_1702_08521_gb300 import vlasov as V

from gpu_helpers import both, from_gpu, rel_l1, rel_max, to_gpu
from test_oracle_vp import fit_damping, landau_root

pytestmark = pytest.mark.gpu


def run_pair(cfg, precision, steps, diag=False, f0=None):
    import torch
    sim, og = both(cfg["grid"], precision)
    kind, params = cfg["ic"]
    f_o = O.init_f(og, kind, params) if f0 is None else f0.copy()
    if precision == V.VP_F32:
        f_o = f_o.astype(np.float32).astype(np.float64)
    to_gpu(sim, f_o)
    _, _, acc = O.field(og, f_o)
    acc = np.ascontiguousarray(acc)
    sim.field()
    d_dev = torch.zeros(steps * V.VP_NDIAG, dtype=torch.float64, device="cuda") if diag else None
    sim.step(cfg["dt"], steps, split=cfg["split"], mode=1, diag=d_dev)
    d_o = O.step(og, f_o, cfg["dt"], steps, acc, split=cfg["split"], mode=1, diag=diag)
    f_g = from_gpu(sim)
    out = dict(f_g=f_g, f_o=f_o, acc_g=sim.accel.cpu().numpy(), acc_o=acc.reshape(-1))
    if diag:
        out["d_g"] = d_dev.cpu().numpy().reshape(steps, V.VP_NDIAG)
        out["d_o"] = d_o
    sim.close()
    return out


def test_landau_fp64_step_parity():
    """One KDK step of the linear Landau configuration (FP64): 1e-12."""
    r = run_pair(inputs.landau_linear(), V.VP_F64, 1)
    assert rel_max(r["f_g"], r["f_o"]) <= 1e-12
    assert rel_max(r["acc_g"], r["acc_o"]) <= 1e-11


def test_landau_fp64_full_run_and_damping():
    """Linear Landau (Nx=64, Nv=128, MP5+PP, dt=0.1, 200 steps) in FP64 on the
    GPU: the run matches the oracle and the measured damping rate and
    frequency match the dispersion relation."""
    cfg = inputs.landau_linear()
    r = run_pair(cfg, V.VP_F64, cfg["steps"], diag=True)
    assert rel_l1(r["f_g"], r["f_o"]) <= 1e-10
    assert np.abs(r["d_g"] - r["d_o"]).max() <= 1e-9 * np.abs(r["d_o"]).max()
    # the damping measured from the GPU's own field history
    sim, og = both(cfg["grid"], V.VP_F64)
    V.vp_init_f(sim.ctx, *cfg["ic"])
    d0 = V.vp_diagnostics(sim.ctx, 1)
    t = cfg["dt"] * np.arange(cfg["steps"] + 1)
    amp = np.concatenate([[d0["mode_amp"]], r["d_g"][:, 6]])
    gamma, omega, _ = fit_damping(t, amp)
    wr, wi = landau_root(0.5)
    assert gamma == pytest.approx(wi, rel=0.03)
    assert omega == pytest.approx(wr, rel=0.01)
    sim.close()


def test_dkd_3d3v_fp64_parity():
    cfg = inputs.plummer(nx=6, nv=8)
    cfg["dt"] = 0.1
    r = run_pair(cfg, V.VP_F64, 2)
    assert rel_max(r["f_g"], r["f_o"]) <= 1e-11


@pytest.mark.parametrize("which", ["landau_nonlinear", "two_stream"])
def test_fp32_run_vs_fp64_oracle(which):
    """FP32 GPU run vs FP64 oracle over 200 steps of the nonlinear 1D1V
    problems on a 64 x 256 grid: relative L1 within 1e-5."""
    cfg = getattr(inputs, which)(64, 256)
    r = run_pair(cfg, V.VP_F32, 200)
    err = rel_l1(r["f_g"], r["f_o"])
    assert err <= 1e-5, err
    assert r["f_g"].min() >= 0.0

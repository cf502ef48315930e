"""GPU parity of the velocity moment, the Poisson solver, the diagnostics and
initial conditions against the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1702_08521_gb300 import inputs
from paper_1702_08521_gb300 import vlasov as V

from gpu_helpers import both, from_gpu, rel_max, to_gpu

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("precision", [V.VP_F32, V.VP_F64])
@pytest.mark.parametrize("dims,nx,nv", [(1, [33], [130]), (2, [6, 5], [12, 20]), (3, [3, 4, 2], [8, 6, 10])])
def test_density_moment(precision, dims, nx, nv):
    g = dict(dims=dims, nx=nx, nv=nv, xlo=[0.0] * dims, xhi=[1.0] * dims, vlo=[-2.0] * dims,
             vhi=[3.0] * dims)
    sim, og = both(g, precision)
    f0 = inputs.random_f(og.NX * og.NV, seed=2).astype(np.float32).astype(np.float64)
    to_gpu(sim, f0)
    V.vp_density_moment(sim.ctx, sim.rho)
    sim.sync()
    rho_g = sim.rho.cpu().numpy()
    rho_o = O.density_moment(og, f0)
    assert rel_max(rho_g, rho_o) <= 1e-13
    sim.close()


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("dims,nx", [(1, [64]), (1, [48]), (2, [16, 12]), (3, [8, 6, 4])])
def test_periodic_poisson(order, dims, nx):
    g = dict(dims=dims, nx=nx, nv=[1] * dims, xlo=[0.0] * dims, xhi=[2.0 + d for d in range(dims)],
             vlo=[-1.0] * dims, vhi=[1.0] * dims, pois_order=order, coupling=-1.0, rho_bg=1.0)
    sim, og = both(g, V.VP_F64)
    rng = np.random.default_rng(order)
    rho = 1.0 + 0.3 * rng.standard_normal(og.NX)
    acc = np.zeros(dims * og.NX)
    phi = np.zeros(og.NX)
    r_t, p_t, a_t = _t(rho), _t(phi), _t(acc)
    V.vp_poisson_solve(sim.ctx, r_t, p_t, a_t)
    sim.sync()
    phi_o, acc_o = O.poisson_solve(og, rho)
    assert rel_max(p_t.cpu().numpy(), phi_o) <= 1e-12
    assert rel_max(a_t.cpu().numpy(), acc_o.reshape(-1)) <= 1e-12
    sim.close()


@pytest.mark.parametrize("n", [6, 8])
def test_isolated_poisson(n):
    h = 0.5
    g = dict(dims=3, nx=[n] * 3, nv=[1] * 3, xlo=[0.0] * 3, xhi=[n * h] * 3, vlo=[-1.0] * 3,
             vhi=[1.0] * 3, poisson=V.VP_POIS_ISOLATED, pois_order=6, coupling=4 * math.pi, rho_bg=0.0)
    sim, og = both(g, V.VP_F64)
    rho = np.random.default_rng(n).random(og.NX)
    p_t, a_t = _t(np.zeros(og.NX)), _t(np.zeros(3 * og.NX))
    V.vp_poisson_solve(sim.ctx, _t(rho), p_t, a_t)
    sim.sync()
    phi_o, acc_o = O.poisson_solve(og, rho)
    assert rel_max(p_t.cpu().numpy(), phi_o) <= 1e-12
    assert rel_max(a_t.cpu().numpy(), acc_o.reshape(-1)) <= 1e-12
    sim.close()


@pytest.mark.parametrize("cfg", [inputs.landau_linear(), inputs.two_stream(32, 64),
                                 inputs.plummer(6, 8)])
def test_initial_conditions_and_diagnostics(cfg):
    prec = V.VP_F64
    sim, og = both(cfg["grid"], prec)
    kind, params = cfg["ic"]
    V.vp_init_f(sim.ctx, kind, params)
    f_g = from_gpu(sim)
    f_o = O.init_f(og, kind, params)
    assert rel_max(f_g, f_o) <= 1e-13
    d_g = V.vp_diagnostics(sim.ctx, 1)
    d_o = O.diagnostics(og, f_o, 1)
    for k in O.DIAG_NAMES:
        assert d_g[k] == pytest.approx(d_o[k], rel=1e-11, abs=1e-14 * (1 + abs(d_o["mass"]))), k
    sim.close()


@pytest.mark.parametrize("cfg", [inputs.two_stream(32, 64), inputs.plummer(6, 8)])
def test_fp32_diagnostics_match_oracle_on_evolved_state(cfg):
    """FP32 f: the moments, energies, extrema and norms (FP64 sums of the FP32
    cells, compensated FP32 partial sums in the velocity moment) against the
    oracle's FP64 diagnostics of the same FP32-rounded state, after a few
    steps so that the state is not an analytic one."""
    sim, og = both(cfg["grid"], V.VP_F32)
    kind, params = cfg["ic"]
    V.vp_init_f(sim.ctx, kind, params)
    sim.field()
    sim.step(cfg["dt"], 3, split=cfg["split"])
    f_g = from_gpu(sim)
    d_g = V.vp_diagnostics(sim.ctx, 1)
    d_o = O.diagnostics(og, f_g, 1)
    for k in O.DIAG_NAMES:
        assert d_g[k] == pytest.approx(d_o[k], rel=1e-9, abs=1e-12 * (1 + abs(d_o["mass"]))), k
    sim.close()


def test_diagnostics_flags_nonfinite():
    g = dict(dims=1, nx=[8], nv=[8], xlo=[0.0], xhi=[1.0], vlo=[-1.0], vhi=[1.0])
    sim, _ = both(g, V.VP_F32)
    f = np.ones(64)
    f[5] = np.nan
    to_gpu(sim, f)
    with pytest.raises(V.VpError) as e:
        V.vp_diagnostics(sim.ctx)
    assert e.value.code == V.VP_ENONFINITE
    sim.close()

"""RK-MPP5 (Sec. 2.1.1, Eqs. 8-10) through the C ABI against the oracle:
drift and kick sweeps on ragged grids (FP64 and FP32), a run of KDK steps of
linear Landau damping, the grid checks, and the CFL bound |nu| < 1/2 that the
device reports through the context's status word."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1702_08521_gb300 import inputs
from paper_1702_08521_gb300 import vlasov as V

from gpu_helpers import accel_tensor, both, from_gpu, rel_l1, rel_max, to_gpu

pytestmark = pytest.mark.gpu

CASES = [
    (1, [37], [45]),
    (1, [64], [130]),
    (1, [6], [1024]),  # long contiguous lines
    (2, [9, 7], [10, 12]),
    (3, [5, 6, 4], [6, 5, 8]),
]


def rk_grid(dims, nx, nv, **kw):
    xhi = [2.0 + 0.37 * d for d in range(dims)]
    return dict(dims=dims, nx=nx, nv=nv, xlo=[0.0] * dims, xhi=xhi,
                vlo=[-3.0 - 0.5 * d for d in range(dims)], vhi=[2.5 + 0.25 * d for d in range(dims)],
                order=5, scheme=V.VP_SCHEME_RK, **kw)


def _dt(og, kick, d, acc):
    """A time step with |nu| = 0.45 on the fastest line of the sweep."""
    if kick:
        dv = (og.vhi[d] - og.vlo[d]) / og.nv[d]
        return 0.45 * dv / np.abs(acc[d]).max()
    dx = (og.xhi[d] - og.xlo[d]) / og.nx[d]
    return 0.45 * dx / np.abs(og.v_centres(d)).max()


@pytest.mark.parametrize("dims,nx,nv", CASES)
@pytest.mark.parametrize("precision", [V.VP_F64, V.VP_F32])
def test_rk_sweeps_match_oracle(dims, nx, nv, precision):
    g = rk_grid(dims, nx, nv)
    sim, og = both(g, precision)
    f0 = inputs.random_f(og.NX * og.NV, seed=17, zeros=0.3)
    if precision == V.VP_F32:
        f0 = f0.astype(np.float32).astype(np.float64)
    acc = inputs.random_accel(og.NX, dims, seed=18, amax=5.0)
    for kick in (0, 1):
        for d in range(dims):
            f_o = f0.copy()
            to_gpu(sim, f0)
            dt = _dt(og, kick, d, acc) * (1 if d % 2 == 0 else -1)
            if kick:
                O.kick_sweep_rk(og, f_o, d, dt, acc[d])
                V.vp_kick_sweep(sim.ctx, d, dt, accel_tensor(sim, acc[d]))
            else:
                O.drift_sweep_rk(og, f_o, d, dt)
                V.vp_drift_sweep(sim.ctx, d, dt)
            f_g = from_gpu(sim)
            if precision == V.VP_F64:
                assert rel_max(f_g, f_o) <= 1e-12, (kick, d, rel_max(f_g, f_o))
            else:
                assert rel_l1(f_g, f_o) <= 5e-6, (kick, d, rel_l1(f_g, f_o))
            assert f_g.min() >= 0.0
    sim.close()


def test_rk_landau_run_matches_oracle():
    """Linear Landau damping (Sec. 3.3 setup, 64 x 128, FP64) with RK-MPP5:
    20 KDK steps of dt = 0.01 (|nu| <= 0.31; the SL run's dt = 0.1 gives 3.0)
    on the GPU against the oracle's sweeps composed in the same order (kicks
    dt/2, drift dt, field, kicks dt/2)."""
    cfg = inputs.landau_linear()
    g = dict(cfg["grid"], scheme=V.VP_SCHEME_RK)
    sim, og = both(g, V.VP_F64)
    f_o = O.init_f(og, *cfg["ic"])
    to_gpu(sim, f_o)
    sim.field()
    dt, steps = 0.01, 20
    sim.step(dt, steps, split=V.VP_SPLIT_KDK)
    _, _, acc = O.field(og, f_o)
    for _ in range(steps):
        O.kick_sweep_rk(og, f_o, 0, 0.5 * dt, acc[0])
        O.drift_sweep_rk(og, f_o, 0, dt)
        _, _, acc = O.field(og, f_o)
        O.kick_sweep_rk(og, f_o, 0, 0.5 * dt, acc[0])
    f_g = from_gpu(sim)
    sim.close()
    assert rel_max(f_g, f_o) <= 1e-11, rel_max(f_g, f_o)


def test_rk_grid_checks():
    with pytest.raises(V.VpError) as e:
        V.Simulation(rk_grid(1, [16], [16], **{}) | {"order": 7}, precision=V.VP_F64)
    assert e.value.code == V.VP_ENOTSUP
    with pytest.raises(V.VpError) as e:
        V.Simulation(rk_grid(1, [16], [16]) | {"scheme": 2}, precision=V.VP_F64)
    assert e.value.code == V.VP_EINVAL


def test_rk_cfl_violation_is_reported():
    """A drift with |nu| = 0.6 on the fastest line: the launch succeeds, the
    shift table flags the CFL bound, and vp_sync reports VP_ECFL."""
    g = rk_grid(1, [32], [16])
    sim, og = both(g, V.VP_F64)
    to_gpu(sim, inputs.random_f(og.NX * og.NV, seed=2))
    dx = (og.xhi[0] - og.xlo[0]) / og.nx[0]
    V.vp_drift_sweep(sim.ctx, 0, 0.6 * dx / np.abs(og.v_centres(0)).max())
    with pytest.raises(V.VpError) as e:
        sim.sync()
    assert e.value.code == V.VP_ECFL
    # the status word is cleared: the context stays usable
    V.vp_drift_sweep(sim.ctx, 0, 0.3 * dx / np.abs(og.v_centres(0)).max())
    sim.sync()
    sim.close()


@pytest.mark.parametrize("dims,nx,nv", [CASES[0], CASES[1], CASES[3], CASES[4]])
def test_rk_two_line_kernel_gives_the_same_bits(dims, nx, nv):
    """FP32 strided RK sweeps walk two lines per thread with the packed pair
    arithmetic unless the one-line kernels are requested; every sweep kind
    gives the same bits both ways (lines of both directions in one tile)."""
    g = rk_grid(dims, nx, nv)
    f0 = inputs.random_f(int(np.prod(nx)) * int(np.prod(nv)), seed=44).astype(np.float32).astype(np.float64)
    acc = inputs.random_accel(int(np.prod(nx)), dims, seed=45, amax=4.0)
    out = []
    for impl in (0, 1):
        sim, og = both(g, V.VP_F32)
        V.vp_set_option(sim.ctx, V.VP_OPT_SWEEP_IMPL, impl)
        res = []
        for kick in (0, 1):
            for d in range(dims):
                to_gpu(sim, f0)
                dt = _dt(og, kick, d, acc)
                if kick:
                    V.vp_kick_sweep(sim.ctx, d, dt, accel_tensor(sim, acc[d]))
                else:
                    V.vp_drift_sweep(sim.ctx, d, dt)
                res.append(from_gpu(sim))
        out.append(res)
        sim.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)

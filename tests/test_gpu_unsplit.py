"""GPU parity of the unsplit step in physical space (Test-1d, reading R23)
against the FP64 oracle, through the C ABI.  FP64 steps agree to 1e-12
relative; FP32 within 4e-6 relative L1 per step (one rounding of f plus the
FP32 arithmetic of two increments).  Ragged tiles along x1, x2 and v, tiny
periodic boxes (fewer cells than the halo), zero-inflow boxes, integer parts
of the shift up to 4 cells, odd and even step counts (the ping-pong ends in f
either way), the argument checks, and sampled cells of the full-size 4096^2 x 2^2
Test-1d grid, each recomputed by the oracle from the two lines through it."""
import numpy as np
import pytest

import oracle as O
from paper_1702_08521_gb300 import inputs
from paper_1702_08521_gb300 import vlasov as V

from gpu_helpers import both, from_gpu, rel_l1, rel_max, to_gpu

pytestmark = pytest.mark.gpu


def vp_grid(nx, nv, vlo, vhi, xbc=O.BC_PERIODIC, order=7, **kw):
    return dict(dims=2, nx=nx, nv=nv, xlo=[0.0, 0.0], xhi=[1.0, 1.3], vlo=vlo, vhi=vhi, xbc=xbc,
                order=order, **kw)


# (grid, dt): Test-1d grids at nu = 0.02 and larger shifts, 2D2V boxes
CASES = [
    (inputs.advect_2d(37, 1, n2=23)["grid"], 0.02 / 37),          # one ragged tile
    (inputs.advect_2d(130, 1, n2=70)["grid"], 0.3 / 130),         # several tiles, nu = 0.3
    (inputs.advect_2d(5, 1, n2=3)["grid"], 2.6 / 5),              # box smaller than the halo, shift 2.6
    (vp_grid([9, 11], [8, 8], [-3.0, -2.0], [3.0, 2.5]), 0.17),   # 2D2V, integer parts up to 4
    (vp_grid([13, 17], [2, 3], [-1.0, -2.0], [1.5, 2.0]), 0.05),  # few velocities, small shifts
    (vp_grid([20, 12], [6, 7], [-2.0, -1.0], [2.0, 1.0], xbc=O.BC_OUTFLOW), 0.1),
    (vp_grid([16, 40], [1, 1], [-1.4, -0.9], [-0.6, -0.1], xbc=O.BC_OUTFLOW, order=5), 0.011),
    (inputs.advect_2d(200, 1, n2=150, nv=2)["grid"], 0.1 / 200),  # interior tiles (contiguous rows)
]


def _scratch(sim):
    import torch
    return torch.empty_like(sim.f)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("nsteps", [1, 2, 3])
def test_unsplit_fp64_matches_oracle(case, nsteps):
    g, dt = CASES[case]
    sim, og = both(g, V.VP_F64)
    f = inputs.random_f(og.NX * og.NV, seed=31 + case)
    to_gpu(sim, f)
    V.vp_drift_unsplit(sim.ctx, dt, nsteps, _scratch(sim))
    for _ in range(nsteps):
        O.drift_unsplit(og, f, dt)
    assert rel_max(from_gpu(sim), f) <= 1e-12
    sim.close()


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("mp,pp", [(1, 1), (0, 0), (1, 0)])
def test_unsplit_fp32_matches_oracle(case, mp, pp):
    g, dt = CASES[case]
    g = {**g, "mp": mp, "pp": pp}
    sim, og = both(g, V.VP_F32)
    f0 = inputs.random_f(og.NX * og.NV, seed=7 + case).astype(np.float32).astype(np.float64)
    to_gpu(sim, f0)
    V.vp_drift_unsplit(sim.ctx, dt, 1, _scratch(sim))
    O.drift_unsplit(og, f0, dt)
    assert rel_l1(from_gpu(sim), f0) <= 4e-6
    sim.close()


def test_unsplit_equals_split_on_the_test1d_sine():
    """Sum-separable data (Eq. 66): unsplit and split steps agree (the oracle
    pins why); here both run on the GPU in FP64 for 50 steps at nu = 0.02."""
    g = inputs.advect_2d(64, 1)["grid"]
    su, og = both(g, V.VP_F64)
    ss, _ = both(g, V.VP_F64)
    f = O.init_f(og, O.IC_ADVECT, [1.0])
    to_gpu(su, f)
    to_gpu(ss, f)
    dt = 0.02 / 64
    V.vp_drift_unsplit(su.ctx, dt, 50, _scratch(su))
    for _ in range(50):
        V.vp_drift_sweep(ss.ctx, 1, dt)
        V.vp_drift_sweep(ss.ctx, 0, dt)
    assert rel_max(from_gpu(su), from_gpu(ss)) <= 1e-13
    su.close()
    ss.close()


def test_unsplit_rectangle_stays_in_range_at_the_papers_cfl():
    """Test-1d rectangle (Eq. 65) on the GPU in FP32, N = 128, nu = 0.02 to
    t = 0.25: within [0, 1] (to FP32 rounding) and mass kept."""
    g = inputs.advect_2d(128, 0)["grid"]
    sim, og = both(g, V.VP_F32)
    V.vp_init_f(sim.ctx, *inputs.advect_2d(128, 0)["ic"])
    m0 = float(sim.f.double().sum())
    dt = 0.02 / 128
    V.vp_drift_unsplit(sim.ctx, dt, int(round(0.25 / dt)), _scratch(sim))
    f = from_gpu(sim)
    assert f.min() >= -1e-6 and f.max() <= 1.0 + 1e-6
    assert abs(f.sum() - m0) <= 1e-5 * m0
    sim.close()


def test_unsplit_argument_checks():
    import torch
    g, dt = CASES[0]
    sim, og = both(g, V.VP_F32)
    f0 = inputs.random_f(og.NX * og.NV, seed=3).astype(np.float32)
    to_gpu(sim, f0.astype(np.float64))
    sc = _scratch(sim)
    for bad, code in ((lambda: V.vp_drift_unsplit(sim.ctx, dt, 1, None), V.VP_EINVAL),
                      (lambda: V.vp_drift_unsplit(sim.ctx, dt, 1, sim.f), V.VP_EINVAL),
                      (lambda: V.vp_drift_unsplit(sim.ctx, dt, -1, sc), V.VP_EINVAL),
                      (lambda: V.vp_drift_unsplit(sim.ctx, float("nan"), 1, sc), V.VP_EINVAL),
                      (lambda: V.vp_drift_unsplit(sim.ctx, 6.0 / 37, 1, sc), V.VP_ENOTSUP)):  # 6 cells
        with pytest.raises(V.VpError) as e:
            bad()
        assert e.value.code == code
    big = torch.empty(sim.f.numel() + 8, dtype=sim.f.dtype, device=sim.f.device)
    with pytest.raises(V.VpError) as e:
        V.vp_drift_unsplit(sim.ctx, dt, 1, big.data_ptr() + 4)  # misaligned
    assert e.value.code == V.VP_EINVAL
    V.vp_drift_unsplit(sim.ctx, dt, 0, sc)  # no step: f unchanged
    assert np.array_equal(from_gpu(sim), f0.astype(np.float64))
    sim.close()
    for dims in (1, 3):
        g1 = dict(dims=dims, nx=[8] * dims, nv=[4] * dims, xlo=[0.0] * dims, xhi=[1.0] * dims,
                  vlo=[-1.0] * dims, vhi=[1.0] * dims)
        s1 = V.Simulation(g1, precision=V.VP_F32)
        with pytest.raises(V.VpError) as e:
            V.vp_drift_unsplit(s1.ctx, 0.01, 1, _scratch(s1))
        assert e.value.code == V.VP_ENOTSUP
        s1.close()
    srk = V.Simulation({**CASES[0][0], "order": 5, "scheme": V.VP_SCHEME_RK}, precision=V.VP_F32)
    with pytest.raises(V.VpError) as e:
        V.vp_drift_unsplit(srk.ctx, dt, 1, _scratch(srk))
    assert e.value.code == V.VP_ENOTSUP
    srk.close()


def test_unsplit_full_size_sampled_cells():
    """The benchmark's HBM-bound unsplit workload (Test-1d sine on 4096^2
    cells with a 2 x 2 velocity grid, FP32, MP7, nu = 0.02 at c_x = 1), one
    step: 64 sampled cells recomputed by the oracle from the x1 and x2 lines
    through each (f + (A_1 f - f) + (A_2 f - f) at that cell, each line at its
    own velocity); and mass kept over the whole grid."""
    n, nv = 4096, 2
    cfg = inputs.advect_2d(n, 1, nv=nv)
    sim = V.Simulation(cfg["grid"], precision=V.VP_F32)
    V.vp_init_f(sim.ctx, *cfg["ic"])
    f0 = sim.f.clone()
    m0 = float(f0.double().sum())
    dt = 0.02 / n
    V.vp_drift_unsplit(sim.ctx, dt, 1, _scratch(sim))
    sim.sync()
    f1 = sim.f.view(n, n, nv * nv)
    a = f0.view(n, n, nv * nv)
    cx = [0.75, 1.25]
    cy = [0.25, 0.75]
    rng = np.random.default_rng(17)
    cells = np.stack([rng.integers(0, n, 64), rng.integers(0, n, 64), rng.integers(0, nv * nv, 64)], axis=1)
    cells[0] = (0, 0, 0)
    cells[1] = (n - 1, n - 1, nv * nv - 1)
    for i, j, v in cells:
        col = a[:, j, v].double().cpu().numpy()
        row = a[i, :, v].double().cpu().numpy()
        a1 = O.advect_line(col, cx[v // nv] * dt * n)[i]
        a2 = O.advect_line(row, cy[v % nv] * dt * n)[j]
        c = col[i]
        want = c + ((a1 - c) + (a2 - c))
        assert abs(float(f1[i, j, v]) - want) <= 6e-7 * max(abs(want), 1.0), (i, j, v)
    assert abs(float(sim.f.double().sum()) - m0) <= 1e-6 * m0
    sim.close()


@pytest.mark.parametrize("precision", [V.VP_F64, V.VP_F32])
def test_unsplit_negative_cells_take_the_theta_form(precision):
    """The unsplit step can leave cells below zero; next to such a cell the PP
    limiter is the paper's theta blend (Eqs. 15-23), which the clamp the split
    sweeps use equals only for non-negative cells.  Input with a fifth of the
    cells negative, one step against the oracle."""
    g, dt = CASES[1]
    sim, og = both(g, precision)
    rng = np.random.default_rng(77)
    f = inputs.random_f(og.NX * og.NV, seed=5)
    f[rng.random(f.size) < 0.2] *= -0.3
    if precision == V.VP_F32:
        f = f.astype(np.float32).astype(np.float64)
    to_gpu(sim, f)
    V.vp_drift_unsplit(sim.ctx, dt, 1, _scratch(sim))
    O.drift_unsplit(og, f, dt)
    if precision == V.VP_F64:
        assert rel_max(from_gpu(sim), f) <= 1e-12
    else:
        assert rel_l1(from_gpu(sim), f) <= 4e-6
    sim.close()


@pytest.mark.parametrize("precision", [V.VP_F64, V.VP_F32])
def test_unsplit_tile_shape_does_not_change_bits(precision):
    """The autotuner (every candidate tile shape launched f -> scratch once,
    f untouched) and the fixed default shape give the same bits: every cell's
    increments are the same walks whatever the tile."""
    g, dt = CASES[1]
    out = []
    for tune in (0, 1):
        sim, og = both(g, precision)
        V.vp_set_option(sim.ctx, V.VP_OPT_AUTOTUNE, tune)
        f = inputs.random_f(og.NX * og.NV, seed=12)
        to_gpu(sim, f)
        V.vp_drift_unsplit(sim.ctx, dt, 3, _scratch(sim))
        out.append(from_gpu(sim))
        sim.close()
    assert np.array_equal(out[0], out[1])

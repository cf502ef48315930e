"""GPU parity of the advection sweeps against the FP64 oracle (through the
C ABI).  FP64 sweeps must agree to 1e-12 relative per sweep; FP32 sweeps
within 2e-6 relative L1 per sweep (single rounding of f plus FP32
arithmetic); integer shifts are exact; f >= 0 is kept exactly."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1702_08521_gb300 import inputs
from paper_1702_08521_gb300 import vlasov as V

from gpu_helpers import accel_tensor, both, from_gpu, rel_l1, rel_max, to_gpu

pytestmark = pytest.mark.gpu


def grid(dims, nx, nv, **kw):
    xhi = [2.0 + 0.37 * d for d in range(dims)]
    return dict(dims=dims, nx=nx, nv=nv, xlo=[0.0] * dims, xhi=xhi,
                vlo=[-3.0 - 0.5 * d for d in range(dims)], vhi=[2.5 + 0.25 * d for d in range(dims)],
                **kw)


CASES = [
    # ragged sizes spanning several tiles along both the line and across lines
    (1, [37], [45]),
    (1, [64], [130]),
    (1, [300], [33]),
    (1, [6], [1024]),  # long contiguous lines: few lines per CTA, many segments
    (1, [4096], [20]),  # long strided lines (the 4096-cell limit): tiles narrower than a warp
    (2, [9, 7], [10, 12]),
    (2, [16, 5], [33, 8]),
    (3, [5, 6, 4], [6, 5, 8]),
]


@pytest.mark.parametrize("dims,nx,nv", CASES)
@pytest.mark.parametrize("order", [5, 7])
@pytest.mark.parametrize("xbc", [0, 1])
def test_fp64_sweeps_match_oracle(dims, nx, nv, order, xbc):
    g = grid(dims, nx, nv, order=order, xbc=xbc)
    sim, og = both(g, V.VP_F64)
    f0 = inputs.random_f(og.NX * og.NV, seed=17 + dims)
    NX = og.NX
    acc = inputs.random_accel(NX, dims, seed=5, amax=7.0)
    rng = np.random.default_rng(3)
    for rep in range(2):
        for kick in (0, 1):
            for d in range(dims):
                dt = float(rng.uniform(-0.9, 0.9))
                f_o = f0.copy()
                to_gpu(sim, f0)
                if kick:
                    O.kick_sweep(og, f_o, d, dt, acc[d])
                    V.vp_kick_sweep(sim.ctx, d, dt, accel_tensor(sim, acc[d]))
                else:
                    O.drift_sweep(og, f_o, d, dt)
                    V.vp_drift_sweep(sim.ctx, d, dt)
                f_g = from_gpu(sim)
                assert rel_max(f_g, f_o) <= 1e-12, (kick, d, dt, rel_max(f_g, f_o))
    sim.close()


TMA_CASES = [
    # every strided sweep eligible for the TMA kernel (inner % 4 == 0), with
    # ragged column tiles and lines up to the 256-cell box limit
    (1, [37], [132]),
    (1, [256], [36]),
    (2, [9, 7], [12, 20]),
    (3, [5, 3, 4], [8, 4, 12]),
]


@pytest.mark.parametrize("dims,nx,nv", TMA_CASES)
@pytest.mark.parametrize("impl", [1, 2, 3])
@pytest.mark.parametrize("precision", [V.VP_F64, V.VP_F32])
def test_sweep_kernels_agree_with_oracle(dims, nx, nv, impl, precision):
    """The strided-axis kernels (staged loads, TMA pipeline, staged loads with
    two lines per thread) against the oracle, with the autotuner on (it must
    leave f untouched)."""
    g = grid(dims, nx, nv, order=7, xbc=1 if dims == 3 else 0)
    sim, og = both(g, precision)
    V.vp_set_option(sim.ctx, V.VP_OPT_SWEEP_IMPL, impl)
    f0 = inputs.random_f(og.NX * og.NV, seed=23).astype(np.float32).astype(np.float64)
    acc = inputs.random_accel(og.NX, dims, seed=8, amax=6.0)
    tol_max = 1e-12 if precision == V.VP_F64 else None
    for kick in (0, 1):
        for d in range(dims):
            f_o = f0.copy()
            to_gpu(sim, f0)
            if kick:
                O.kick_sweep(og, f_o, d, 0.53, acc[d])
                V.vp_kick_sweep(sim.ctx, d, 0.53, accel_tensor(sim, acc[d]))
            else:
                O.drift_sweep(og, f_o, d, 0.71)
                V.vp_drift_sweep(sim.ctx, d, 0.71)
            f_g = from_gpu(sim)
            if tol_max:
                assert rel_max(f_g, f_o) <= tol_max, (kick, d)
            else:
                assert rel_l1(f_g, f_o) <= 2e-6, (kick, d)
            tu = V.vp_get_tuning(sim.ctx, kick, d)
            assert tu["impl"] in (1, 2, 3)
            if impl == 1:
                assert tu["impl"] == 1
    sim.close()


@pytest.mark.parametrize("mp,pp", [(0, 0), (1, 0), (0, 1)])
def test_fp64_limiter_switches(mp, pp):
    g = grid(2, [12, 9], [20, 17], order=7, mp=mp, pp=pp)
    sim, og = both(g, V.VP_F64)
    f0 = inputs.random_f(og.NX * og.NV, seed=99)
    for d in range(2):
        f_o = f0.copy()
        to_gpu(sim, f0)
        O.drift_sweep(og, f_o, d, 0.37)
        V.vp_drift_sweep(sim.ctx, d, 0.37)
        assert rel_max(from_gpu(sim), f_o) <= 1e-12
    sim.close()


@pytest.mark.parametrize("dims,nx,nv", CASES[:5])
def test_fp32_sweeps_match_oracle(dims, nx, nv):
    g = grid(dims, nx, nv, order=7)
    sim, og = both(g, V.VP_F32)
    # inputs representable in float so both sides start from the same f
    f0 = inputs.random_f(og.NX * og.NV, seed=7).astype(np.float32).astype(np.float64)
    acc = inputs.random_accel(og.NX, dims, seed=6, amax=5.0)
    for kick in (0, 1):
        for d in range(dims):
            f_o = f0.copy()
            to_gpu(sim, f0)
            if kick:
                O.kick_sweep(og, f_o, d, 0.61, acc[d])
                V.vp_kick_sweep(sim.ctx, d, 0.61, accel_tensor(sim, acc[d]))
            else:
                O.drift_sweep(og, f_o, d, -0.43)
                V.vp_drift_sweep(sim.ctx, d, -0.43)
            f_g = from_gpu(sim)
            assert rel_l1(f_g, f_o) <= 2e-6, (kick, d, rel_l1(f_g, f_o))
            assert f_g.min() >= 0.0
    sim.close()


@pytest.mark.parametrize("precision", [V.VP_F32, V.VP_F64])
def test_integer_shift_is_exact_on_gpu(precision):
    # dyadic box and dt: s = v dt / h is an exact integer for every velocity
    n, nv = 32, 8
    g = dict(dims=1, nx=[n], nv=[nv], xlo=[0.0], xhi=[1.0], vlo=[-4.0], vhi=[4.0], order=7)
    sim, og = both(g, precision)
    f0 = inputs.random_f(n * nv, seed=1).astype(np.float32).astype(np.float64)
    to_gpu(sim, f0)
    # v = -3.5 .. 3.5 step 1; h = 1/32; dt = 1/16 -> s = 2 v: odd integers
    V.vp_drift_sweep(sim.ctx, 0, 1.0 / 16.0)
    f_g = from_gpu(sim).reshape(n, nv)
    v = og.v_centres(0)
    want = np.stack([np.roll(f0.reshape(n, nv)[:, j], int(round(2 * v[j]))) for j in range(nv)], axis=1)
    assert np.array_equal(f_g, want)
    sim.close()


def test_positivity_and_mass_fp32():
    g = grid(2, [24, 20], [40, 36], order=7)
    sim, og = both(g, V.VP_F32)
    f0 = (inputs.random_f(og.NX * og.NV, seed=44, zeros=0.5) ** 6).astype(np.float32)
    to_gpu(sim, f0)
    m0 = float(np.sum(f0, dtype=np.float64))
    for _ in range(5):
        for d in range(2):
            V.vp_drift_sweep(sim.ctx, d, 0.77)
    f_g = from_gpu(sim)
    assert f_g.min() >= 0.0
    assert abs(f_g.sum() - m0) / m0 < 1e-6
    sim.close()


def test_sweep_rejects_bad_arguments():
    g = grid(1, [16], [16])
    sim, _ = both(g, V.VP_F32)
    with pytest.raises(V.VpError):
        V.vp_drift_sweep(sim.ctx, 1, 0.1)
    with pytest.raises(V.VpError):
        V.vp_drift_sweep(sim.ctx, 0, float("nan"))
    with pytest.raises(V.VpError):
        V.vp_kick_sweep(sim.ctx, 0, 0.1, None)
    sim.close()


@pytest.mark.parametrize("dims,nx,nv", [(2, [8, 8], [16, 16]), (1, [64], [96]), (1, [2048], [64])])
def test_sweep_bits_do_not_depend_on_tuning(dims, nx, nv):
    """Every sweep gives the same bits whatever kernel, tile width and
    segment count runs it: each implementation with the default tiles, and
    three independently autotuned contexts (timing-based choices)."""
    L = 4 * math.pi
    g = dict(dims=dims, nx=nx, nv=nv, xlo=[0.0] * dims, xhi=[L] * dims, vlo=[-6.0] * dims, vhi=[6.0] * dims,
             order=7)
    n = int(np.prod(nx)) * int(np.prod(nv))
    f0 = (inputs.random_f(n, seed=21, zeros=0.3) ** 2).astype(np.float32)
    setups = [(0, 0), (1, 0), (2, 0), (3, 0), (0, 1), (0, 1), (1, 1), (3, 1)]  # (sweep impl, autotune)
    sweeps = [(1, d) for d in range(dims)] + [(0, d) for d in range(dims)]
    results = []
    for impl, tune in setups:
        out = []
        for kick, d in sweeps:
            sim, _ = both(g, V.VP_F32)
            V.vp_set_option(sim.ctx, V.VP_OPT_SWEEP_IMPL, impl)
            V.vp_set_option(sim.ctx, V.VP_OPT_AUTOTUNE, tune)
            to_gpu(sim, f0)
            sim.field()
            if kick:
                V.vp_kick_sweep(sim.ctx, d, 0.13, sim.accel[d * sim.NX:])
            else:
                V.vp_drift_sweep(sim.ctx, d, 0.37)
            out.append(from_gpu(sim))
            sim.close()
        results.append(out)
    for out in results[1:]:
        for a, b in zip(out, results[0]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("dims,nx,nv", [(1, [40], [48]), (2, [9, 8], [12, 16])])
def test_fp32_positivity_exact_down_to_subnormals(dims, nx, nv):
    """FP32 cells spread log-uniformly over 1e-45 .. 1 (many subnormal, some
    exactly 0) and lines of subnormals only: after 30 sweeps of every kind with
    random time steps f stays >= 0 exactly (the PP limiter in mass form with
    rounded-down half cells), and the state matches the FP64 oracle run from
    the same FP32 values within the FP32 sweep tolerance."""
    g = grid(dims, nx, nv, order=7, xbc=0)
    sim, og = both(g, V.VP_F32)
    rng = np.random.default_rng(71)
    n = og.NX * og.NV
    f0 = inputs.random_f(n, seed=72) * 10.0 ** rng.uniform(-45, 0, size=n)
    f0 = f0.reshape(og.shape)
    # whole spatial lines of subnormals only
    f0[0] = rng.random(f0[0].shape) * 1e-39
    f0 = f0.reshape(-1).astype(np.float32).astype(np.float64)
    acc = inputs.random_accel(og.NX, dims, seed=73, amax=5.0)
    to_gpu(sim, f0)
    f_o = f0.copy()
    for _ in range(30):
        kick = int(rng.integers(0, 2))
        d = int(rng.integers(0, dims))
        dt = float(rng.uniform(-0.8, 0.8))
        if kick:
            V.vp_kick_sweep(sim.ctx, d, dt, accel_tensor(sim, acc[d]))
            O.kick_sweep(og, f_o, d, dt, acc[d])
        else:
            V.vp_drift_sweep(sim.ctx, d, dt)
            O.drift_sweep(og, f_o, d, dt)
        f_g = from_gpu(sim)
        assert f_g.min() >= 0.0
    assert rel_l1(f_g, f_o) <= 1e-5
    sim.close()

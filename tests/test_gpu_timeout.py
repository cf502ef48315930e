"""Bounded device-side waits give up cleanly: a wait limit of zero makes
every dependency wait of the ensemble kernel, and every tile barrier of the
TMA-fed sweep, run out at once.  The kernel records VP_ETIMEOUT, drains its
own copies and returns; the host reads the status, and the context (or a
fresh ensemble) then runs normally.  Nothing hangs: no wait spins at all."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1702_08521_gb300 import inputs
from paper_1702_08521_gb300 import vlasov as V

from gpu_helpers import both, from_gpu, rel_l1, to_gpu

pytestmark = pytest.mark.gpu


def _specs():
    out = []
    for nx, nv, k in ((32, 64, 0.5), (64, 128, 0.4)):
        out.append(dict(dims=1, nx=[nx], nv=[nv], xlo=[0.0], xhi=[2 * math.pi / k], vlo=[-6.0], vhi=[6.0]))
    return out


def _ensemble(stream):
    import torch
    runs = [V.make_run(**s) for s in _specs()]
    ens = V.vp_ensemble_create(runs, 7, stream)
    pool = torch.zeros(V.vp_ensemble_num_cells(ens) + 64, dtype=torch.float32, device="cuda")
    V.vp_ensemble_bind(ens, pool)
    for i in range(len(runs)):
        V.vp_ensemble_init_run(ens, i, V.VP_IC_LANDAU, [0.1, 0.5, 0.0, 0.0, 1.0, 1.0])
    V.vp_ensemble_field(ens)
    return ens, pool


def test_ensemble_dependency_wait_times_out_and_reports():
    import torch
    stream = torch.cuda.Stream()
    ens, pool = _ensemble(stream)
    V.vp_ensemble_set_wait_limit(ens, 0)
    V.vp_ensemble_step(ens, 0.05, 1)
    with pytest.raises(V.VpError) as e:
        V.vp_ensemble_sync(ens)
    assert e.value.code == V.VP_ETIMEOUT
    # the status word was cleared; with the default limit the same ensemble
    # steps again (its f is undefined after the abandoned step, so the
    # result is checked on a fresh ensemble against the single-run path)
    V.vp_ensemble_set_wait_limit(ens, 1 << 24)
    V.vp_ensemble_step(ens, 0.05, 1)
    V.vp_ensemble_sync(ens)
    V.vp_ensemble_destroy(ens)
    ens2, pool2 = _ensemble(stream)
    V.vp_ensemble_step(ens2, 0.05, 5)
    V.vp_ensemble_sync(ens2)
    s = _specs()[1]
    sim = V.Simulation(dict(s, order=7), precision=V.VP_F32)
    V.vp_init_f(sim.ctx, V.VP_IC_LANDAU, [0.1, 0.5, 0.0, 0.0, 1.0, 1.0])
    sim.field()
    sim.step(0.05, 5, split=V.VP_SPLIT_KDK)
    off, _ = V.vp_ensemble_run_layout(ens2, 1)
    got = pool2[off:off + 64 * 128].double().cpu().numpy()
    assert rel_l1(got, from_gpu(sim)) <= 1e-6
    sim.close()
    V.vp_ensemble_destroy(ens2)


def test_tma_tile_wait_times_out_and_reports():
    g = dict(dims=1, nx=[37], nv=[132], xlo=[0.0], xhi=[2.0], vlo=[-3.0], vhi=[2.5], order=7)
    sim, og = both(g, V.VP_F32)
    V.vp_set_option(sim.ctx, V.VP_OPT_SWEEP_IMPL, 2)
    V.vp_set_option(sim.ctx, V.VP_OPT_AUTOTUNE, 0)
    f0 = inputs.random_f(og.NX * og.NV, seed=4).astype(np.float32).astype(np.float64)
    to_gpu(sim, f0)
    V.vp_set_option(sim.ctx, V.VP_OPT_WAIT_LIMIT, 0)
    V.vp_drift_sweep(sim.ctx, 0, 0.3)
    # only the TMA kernel has a tile barrier that can run out in a plain sweep
    with pytest.raises(V.VpError) as e:
        sim.sync()
    assert e.value.code == V.VP_ETIMEOUT
    # default limit again: the same context sweeps correctly
    V.vp_set_option(sim.ctx, V.VP_OPT_WAIT_LIMIT, 1 << 26)
    to_gpu(sim, f0)
    V.vp_drift_sweep(sim.ctx, 0, 0.3)
    f_o = f0.copy()
    O.drift_sweep(og, f_o, 0, 0.3)
    assert rel_l1(from_gpu(sim), f_o) <= 2e-6
    sim.close()

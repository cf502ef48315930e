"""Batched ensemble (one persistent launch per KDK step of all runs) against
the single-run path (itself checked against the oracle) and the oracle."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1702_08521_gb300 import inputs
from paper_1702_08521_gb300 import vlasov as V

from gpu_helpers import rel_l1

pytestmark = pytest.mark.gpu


def _runs():
    """A small uneven ensemble: 1D Landau / two-stream of several sizes and
    one 2D2V Landau run."""
    specs = []
    for kind, nx, nv, k, a in [("landau", 32, 64, 0.5, 0.3), ("two_stream", 64, 128, 0.4, 0.05),
                               ("landau", 128, 256, 0.35, 0.01), ("landau", 256, 512, 0.6, 0.2),
                               ("two_stream", 32, 512, 0.3, 0.1)]:
        vmax = 6.0 if kind == "landau" else 8.0
        specs.append(dict(kind=kind, dims=1, nx=[nx], nv=[nv], k=[k], alpha=a, xlo=[0.0],
                          xhi=[2 * math.pi / k], vlo=[-vmax], vhi=[vmax]))
    specs.append(dict(kind="landau", dims=2, nx=[16, 16], nv=[32, 32], k=[0.5, 0.5], alpha=0.05,
                      xlo=[0.0, 0.0], xhi=[4 * math.pi] * 2, vlo=[-6.0, -6.0], vhi=[6.0, 6.0]))
    return specs


def _ic(spec):
    if spec["kind"] == "landau":
        k = spec["k"] + [0.0] * (3 - len(spec["k"]))
        return V.VP_IC_LANDAU, [spec["alpha"], k[0], k[1], k[2], 1.0, 1.0]
    return V.VP_IC_TWOSTREAM, [spec["alpha"], spec["k"][0]]


def _grid(spec):
    return dict(dims=spec["dims"], nx=spec["nx"], nv=spec["nv"], xlo=spec["xlo"], xhi=spec["xhi"],
                vlo=spec["vlo"], vhi=spec["vhi"], order=7)


def _ensemble(specs, stream):
    import torch
    runs = [V.make_run(**_grid(s)) for s in specs]
    ens = V.vp_ensemble_create(runs, 7, stream)
    pool = torch.zeros(V.vp_ensemble_num_cells(ens) + 64, dtype=torch.float32, device="cuda")
    V.vp_ensemble_bind(ens, pool)
    for i, s in enumerate(specs):
        V.vp_ensemble_init_run(ens, i, *_ic(s))
    V.vp_ensemble_field(ens)
    return ens, pool


def _run_slice(ens, pool, i, spec):
    off, _ = V.vp_ensemble_run_layout(ens, i)
    n = int(np.prod(spec["nx"])) * int(np.prod(spec["nv"]))
    return pool[off:off + n].double().cpu().numpy()


def test_ensemble_matches_single_runs():
    import torch
    specs = _runs()
    stream = torch.cuda.Stream()
    ens, pool = _ensemble(specs, stream)
    dt, steps = 0.05, 20
    V.vp_ensemble_step(ens, dt, steps)
    V.vp_ensemble_sync(ens)
    for i, s in enumerate(specs):
        sim = V.Simulation(_grid(s), precision=V.VP_F32)
        V.vp_init_f(sim.ctx, *_ic(s))
        sim.field()
        sim.step(dt, steps, split=V.VP_SPLIT_KDK)
        sim.sync()
        ref = sim.f.double().cpu().numpy()
        got = _run_slice(ens, pool, i, s)
        assert rel_l1(got, ref) <= 1e-6, (i, rel_l1(got, ref))
        assert got.min() >= 0.0
        sim.close()
    V.vp_ensemble_destroy(ens)


def test_every_ensemble_member_vs_oracle():
    """Every member of the uneven ensemble (1D1V Landau and two-stream of
    several sizes, and the 2D2V Landau run: its strided and contiguous tiles,
    tiled density and in-CTA 2D Poisson solve), FP32 in the persistent
    kernel, against the FP64 oracle after 20 KDK steps from the same
    FP32-rounded initial state."""
    import torch
    specs = _runs()
    stream = torch.cuda.Stream()
    ens, pool = _ensemble(specs, stream)
    f_init = [_run_slice(ens, pool, i, s) for i, s in enumerate(specs)]
    V.vp_ensemble_step(ens, 0.05, 20)
    V.vp_ensemble_sync(ens)
    for i, s in enumerate(specs):
        og = O.grid(**_grid(s))
        kind, params = _ic(s)
        f = O.init_f(og, kind, params)
        # the ensemble initialised its own f on the device: its t = 0 state is
        # the oracle's, rounded to FP32
        assert rel_l1(f_init[i], f.astype(np.float32).astype(np.float64)) <= 1e-7, i
        f = f_init[i].copy()
        _, _, acc = O.field(og, f)
        O.step(og, f, 0.05, 20, np.ascontiguousarray(acc), split=O.SPLIT_KDK)
        got = _run_slice(ens, pool, i, s)
        assert rel_l1(got, f) <= 1e-5, (i, rel_l1(got, f))
        assert got.min() >= 0.0
    V.vp_ensemble_destroy(ens)


def test_autotune_leaves_f_unchanged_and_graph_matches_direct():
    import torch
    specs = _runs()
    stream = torch.cuda.Stream()
    ens, pool = _ensemble(specs, stream)
    before = pool.clone()
    V.vp_ensemble_autotune(ens, 0.05)  # timed steps from a snapshot, restored
    V.vp_ensemble_sync(ens)
    assert torch.equal(before, pool)
    tiles = V.vp_ensemble_get_tiles(ens)
    assert tiles["W"] in (32, 64, 128) and tiles["ctas_per_sm"] >= 1
    # graph replay (non-default stream) vs direct launches on the legacy stream
    V.vp_ensemble_step(ens, 0.05, 3)
    V.vp_ensemble_sync(ens)
    ens2, pool2 = _ensemble(specs, None)
    V.vp_ensemble_set_tiles(ens2, tiles["W"], tiles["R"], tiles["ctas_per_sm"])
    V.vp_ensemble_step(ens2, 0.05, 3)
    V.vp_ensemble_sync(ens2)
    n = V.vp_ensemble_num_cells(ens)
    assert rel_l1(pool2[:n].double().cpu().numpy(), pool[:n].double().cpu().numpy()) <= 1e-6
    V.vp_ensemble_destroy(ens)
    V.vp_ensemble_destroy(ens2)


@pytest.mark.parametrize("graph", [True, False])
def test_ensemble_follows_a_change_of_dt(graph):
    """Steps at one dt, then at another, then back (the drift shifts come from
    a table made once per dt; a stale one would move every drift by the old
    shift): every member against the single-run path after the same
    sequence, with the step graph (a stream of its own) and with direct
    launches (the legacy stream)."""
    import torch
    specs = _runs()
    stream = torch.cuda.Stream() if graph else None
    ens, pool = _ensemble(specs, stream)
    seq = [(0.05, 4), (0.03, 3), (0.05, 2)]
    for dt, n in seq:
        V.vp_ensemble_step(ens, dt, n)
    V.vp_ensemble_sync(ens)
    for i, s in enumerate(specs):
        sim = V.Simulation(_grid(s), precision=V.VP_F32)
        V.vp_init_f(sim.ctx, *_ic(s))
        sim.field()
        for dt, n in seq:
            sim.step(dt, n, split=V.VP_SPLIT_KDK)
        sim.sync()
        ref = sim.f.double().cpu().numpy()
        got = _run_slice(ens, pool, i, s)
        assert rel_l1(got, ref) <= 1e-6, (i, rel_l1(got, ref))
        sim.close()
    V.vp_ensemble_destroy(ens)


def test_flat_vote_does_not_change_the_bits():
    """The walkers with and without the warp vote on flat stencils give the
    same f, bit for bit (the flux of a flat stencil is its value exactly);
    the setter checks its argument and the tuner leaves a valid choice."""
    import torch
    specs = _runs()
    out = []
    for on in (1, 0):
        ens, pool = _ensemble(specs, torch.cuda.Stream())
        V.vp_ensemble_set_flat_vote(ens, on)
        assert V.vp_ensemble_get_flat_vote(ens) == on
        V.vp_ensemble_step(ens, 0.05, 6)
        V.vp_ensemble_sync(ens)
        out.append(pool[:V.vp_ensemble_num_cells(ens)].clone())
        if on == 0:
            with pytest.raises(V.VpError):
                V.vp_ensemble_set_flat_vote(ens, 2)
            V.vp_ensemble_autotune(ens, 0.05)
            assert V.vp_ensemble_get_flat_vote(ens) in (0, 1)
        V.vp_ensemble_destroy(ens)
    assert torch.equal(out[0], out[1])

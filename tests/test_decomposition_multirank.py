"""The paper's parallel layout (Sec. 2.3) on two CPU ranks over gloo.

Physical space is split into blocks along x1 (one slab of planes per rank),
velocity space is not decomposed.  Per KDK step (Eq. 55): the half kicks and
the x2 drift need only the rank's own planes; before the x1 drift every rank
receives a halo of max|N| + 4 planes from each neighbour (N the integer part
of the largest shift, 4 the reach of the MP7 stencil), advances the lines of
its extended slab with zero beyond the halo, and keeps its own planes; the
density moment is local, the slabs' densities are gathered on every rank and
the Poisson solve is replicated.  Each rank computes with the FP64 oracle; the
gathered result must equal the single-rank oracle run bit for bit.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# 16 x 8 spatial cells of unit width, 8 x 8 velocity cells of unit width: the
# slab grids' cell widths equal the global ones exactly
N1, N2, NV, DT, STEPS = 16, 8, 8, 0.7, 4
IC = [0.2, 2 * np.pi / 16, 2 * np.pi / 8, 0.0, 1.0, 1.0]  # Landau: alpha, k1, k2, k3, sigma, amp


def _global_grid(O):
    return O.grid(2, [N1, N2], [NV, NV], [0.0, 0.0], [float(N1), float(N2)], [-4.0, -4.0], [4.0, 4.0],
                  order=7, coupling=-1.0, rho_bg=1.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = _global_grid(O)
    m = N1 // world                      # planes per rank
    lo = rank * m
    left, right = (rank - 1) % world, (rank + 1) % world
    nvc = NV * NV
    f = O.init_f(g, O.IC_LANDAU, IC).reshape(N1, N2 * nvc)[lo:lo + m].copy()
    # the rank's own slab as a grid (x1 planes lo .. lo + m - 1)
    sg = O.grid(2, [m, N2], [NV, NV], [float(lo), 0.0], [float(lo + m), float(N2)], [-4.0, -4.0], [4.0, 4.0],
                order=7, coupling=-1.0, rho_bg=1.0)
    # halo: the largest integer shift of an x1 line plus the stencil's reach
    v1 = g.v_centres(0)
    H = int(np.max(np.abs(np.round(v1 * DT / 1.0)))) + 4
    assert H <= m
    eg = O.grid(2, [m + 2 * H, N2], [NV, NV], [float(lo - H), 0.0], [float(lo + m + H), float(N2)],
                [-4.0, -4.0], [4.0, 4.0], order=7, xbc=O.BC_OUTFLOW, coupling=-1.0, rho_bg=1.0)

    def field(fs):
        rho = torch.from_numpy(O.density_moment(sg, fs.ravel()))
        parts = [torch.empty_like(rho) for _ in range(world)]
        dist.all_gather(parts, rho)
        _, acc = O.poisson_solve(g, torch.cat(parts).numpy())
        return np.ascontiguousarray(acc.reshape(2, N1, N2)[:, lo:lo + m].reshape(2, m * N2))

    def drift_x1(fs):
        send_l = torch.from_numpy(np.ascontiguousarray(fs[:H]))
        send_r = torch.from_numpy(np.ascontiguousarray(fs[m - H:]))
        halo_l = torch.empty_like(send_r)
        halo_r = torch.empty_like(send_l)
        reqs = [dist.isend(send_l, left, tag=0), dist.isend(send_r, right, tag=1),
                dist.irecv(halo_l, left, tag=1), dist.irecv(halo_r, right, tag=0)]
        for q in reqs:
            q.wait()
        ext = np.ascontiguousarray(np.concatenate([halo_l.numpy(), fs, halo_r.numpy()]))
        O.drift_sweep(eg, ext.reshape(-1), 0, DT)
        return ext[H:H + m].copy()

    acc = field(f)
    for _ in range(STEPS):
        for d in range(2):
            O.kick_sweep(sg, f.reshape(-1), d, 0.5 * DT, acc[d])
        O.drift_sweep(sg, f.reshape(-1), 1, DT)
        f = drift_x1(f)
        acc = field(f)
        for d in range(2):
            O.kick_sweep(sg, f.reshape(-1), d, 0.5 * DT, acc[d])
    slabs = [torch.empty(m, N2 * nvc, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(slabs, torch.from_numpy(f))
    if rank == 0:
        out["f"] = torch.cat(slabs).numpy().reshape(-1).tobytes()
        out["H"] = H
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_spatial_blocks_equal_single_rank_oracle():
    import oracle as O
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    got = np.frombuffer(out["f"], dtype=np.float64)
    assert out["H"] == 6  # |v1| <= 3.5, dt = 0.7: shifts of at most 2 whole cells
    g = _global_grid(O)
    f = O.init_f(g, O.IC_LANDAU, IC)
    _, _, acc = O.field(g, f)
    O.step(g, f, DT, STEPS, np.ascontiguousarray(acc), split=O.SPLIT_KDK)
    assert np.array_equal(got, f)
    assert not np.array_equal(f, O.init_f(g, O.IC_LANDAU, IC))  # the run moved f

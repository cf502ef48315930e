"""Learned flux correction on a coarser velocity grid: data generation from
fine-grid runs of the method, training, and coarse runs with the network.

The correction acts on the spatial sweeps (drifts): on a coarser velocity
grid their error comes from the spread of speeds inside one velocity cell,
which moves the sub-cell velocity gradient of f across x.  The network sees
the spatial stencil of the line and the velocity difference and curvature
from its neighbouring velocity cells at the same positions.  Velocity sweeps (kicks)
run the plain scheme: on these grids their coarse-grid error is orders of
magnitude below the drifts'.

Orchestration only: every arithmetic step (sweeps, fine-flux extraction,
restriction, sample construction, forward/backward, Adam, learned sweeps)
runs in the CUDA library through the C ABI; torch holds device memory and
selects rows (valid samples, minibatches).
"""
from __future__ import annotations

import math

import numpy as np

from . import vlasov as V

NFEAT = 25  # network inputs: 8 stencil values, 8 velocity differences, 8 velocity curvatures, nu


def landau_grid(dims: int, nx: int, nv: int, k: float = 0.5, vmax: float = 6.0) -> dict:
    L = 2 * math.pi / k
    return dict(dims=dims, nx=[nx] * dims, nv=[nv] * dims, xlo=[0.0] * dims, xhi=[L] * dims,
                vlo=[-vmax] * dims, vhi=[vmax] * dims, order=7)


def _landau_ic(dims, k, alpha):
    kk = [k] * dims + [0.0] * (3 - dims)
    return V.VP_IC_LANDAU, [alpha, kk[0], kk[1], kk[2], 1.0, 1.0]


def _sweeps(dims):
    """(kick, dim, dt factor) of a KDK step, with None for the field solve."""
    seq = [(1, d, 0.5) for d in range(dims)] + [(0, d, 1.0) for d in range(dims - 1, -1, -1)]
    return seq + [None] + [(1, d, 0.5) for d in range(dims)]


class Sampler:
    """Builds training pairs for one (fine grid, coarse factor) combination."""

    def __init__(self, dims: int, nx: int, nv_fine: int, factor: int, k: float, stream):
        import torch
        self.torch = torch
        self.dims, self.factor, self.stream = dims, factor, stream
        self.gf = landau_grid(dims, nx, nv_fine, k)
        self.gc = landau_grid(dims, nx, nv_fine // factor, k)
        self.fine = V.Simulation(self.gf, precision=V.VP_F32, stream=stream)
        self.coarse = V.Simulation(self.gc, precision=V.VP_F32, stream=stream)
        self.maps = {}
        for kick in (0, 1):
            for d in range(dims):
                m, ncl, grp = V.vp_fluxnet_line_map(V.make_grid(**self.gf), V.make_grid(**self.gc),
                                                    factor, kick, d)
                self.maps[(kick, d)] = (torch.as_tensor(m, dtype=torch.int64, device="cuda"), ncl, grp)

    def restrict(self):
        nv = self.gf["nv"]
        if self.dims == 2:
            V.vp_restrict_velocity(self.fine.f, self.coarse.f, self.fine.NX, nv[0], nv[1], self.factor,
                                   self.factor, self.stream)
        else:
            V.vp_restrict_velocity(self.fine.f, self.coarse.f, self.fine.NX, nv[0], 1, self.factor, 1,
                                   self.stream)

    def samples(self, kick, d, dt, zmin, keep, rng, importance: float = 0.0):
        """Training pairs of cells for the sweep (kick, d, dt) of the current
        fine state: for every cell of the coarse lines, its left and right
        interfaces (rows 2m, 2m + 1 of X and y) with the coefficients of the
        cell-update residual r = (s_r (g_r - y_r) - s_l (g_l - y_l)) / s_c,
        s_c = max(s_l, s_r), s the stencil maximum of an interface.

        keep: number of cells kept (all when 0), drawn without replacement
        with probability proportional to s_c^importance, so that with
        importance = 2 the mean squared residual weighs cells by the square
        of their mass scale; importance = 0 draws uniformly.
        Returns (X [2n][NFEAT], y [2n], coef [2n])."""
        torch = self.torch
        # everything on the library stream: the acceleration copy below must
        # follow the field solve that wrote it, and the buffers belong there
        with torch.cuda.stream(self.stream):
            acc = self.fine.accel[d * self.fine.NX:] if kick else None
            Lf = self.gf["nv"][d] if kick else self.gf["nx"][d]
            every = self.factor if kick else 1
            nlf = self.fine.NX * int(np.prod(self.gf["nv"])) // Lf
            nout = Lf // every + 1
            Gf = torch.empty(nlf * nout, dtype=torch.float64, device="cuda")
            V.vp_fine_flux(self.fine.ctx, kick, d, dt, acc, every, Gf)
            m, ncl, grp = self.maps[(kick, d)]
            Gc = torch.empty(ncl * nout, dtype=torch.float64, device="cuda")
            V.vp_group_mean(Gf, ncl, nout, m, grp, 1.0 / every, Gc, self.stream)
            self.restrict()
            ns = ncl * nout
            X = torch.empty(ns * NFEAT, dtype=torch.float32, device="cuda")
            y = torch.empty(ns, dtype=torch.float32, device="cuda")
            sc = torch.empty(ns, dtype=torch.float32, device="cuda")
            cacc = self.coarse.accel[d * self.coarse.NX:] if kick else None
            if kick:
                self.coarse.accel.copy_(self.fine.accel)
            V.vp_make_samples(self.coarse.ctx, kick, d, dt, cacc, Gc, zmin, X, y, sc)
            # cells: left interface i, right interface i + 1 (interface 0 again
            # at the end of a periodic line, whose interface L is not sampled)
            Lc = nout - 1
            yl = y.view(ncl, nout)
            right = torch.arange(1, nout, device="cuda").expand(ncl, Lc).clone()
            right[~torch.isfinite(yl[:, Lc]), Lc - 1] = 0
            base = (torch.arange(ncl, device="cuda") * nout).unsqueeze(1)
            li = (base + torch.arange(Lc, device="cuda")).reshape(-1)
            ri = (base + right).reshape(-1)
            ok = torch.isfinite(y[li]) & torch.isfinite(y[ri])
            li, ri = li[ok].contiguous(), ri[ok].contiguous()
            npair = li.numel()
            # the pairs' loss coefficients and draw weights (library kernel)
            coef = torch.empty(2 * npair, dtype=torch.float32, device="cuda")
            wgt = torch.empty(npair, dtype=torch.float64, device="cuda")
            V.vp_pair_coefs(sc, li, ri, npair, importance, coef, wgt, self.stream)
            coef = coef.view(npair, 2)
            if keep and npair > keep:
                # draw on the GPU, seeded from the caller's generator
                gen = torch.Generator(device="cuda")
                gen.manual_seed(int(rng.integers(0, 2 ** 62)))
                nz = int((wgt > 0).sum())
                sel = torch.multinomial(wgt, min(keep, nz), replacement=False, generator=gen)
                li, ri, coef = li[sel], ri[sel], coef[sel]
            idx = torch.stack([li, ri], dim=1).reshape(-1)
            Xv = X.view(ns, NFEAT)[idx]
            yv = y[idx]
            cv = coef.reshape(-1)
        self.stream.synchronize()
        return Xv, yv, cv

    def run_draw(self, k, alpha, dt, steps, every_step, zmin, keep, rng, importance: float = 0.0):
        """Fine run from the Landau state (k, alpha); pairs of its spatial
        sweeps every `every_step` steps."""
        V.vp_init_f(self.fine.ctx, *_landau_ic(self.dims, k, alpha))
        self.fine.field()
        Xs, ys, cs = [], [], []
        for n in range(steps):
            take = (n + 1) % every_step == 0
            for sw in _sweeps(self.dims):
                if sw is None:
                    self.fine.field()
                    continue
                kick, d, fac = sw
                if take and not kick:
                    X, y, c = self.samples(kick, d, fac * dt, zmin, keep, rng, importance)
                    Xs.append(X)
                    ys.append(y)
                    cs.append(c)
                acc = self.fine.accel[d * self.fine.NX:] if kick else None
                if kick:
                    V.vp_kick_sweep(self.fine.ctx, d, fac * dt, acc)
                else:
                    V.vp_drift_sweep(self.fine.ctx, d, fac * dt)
        return Xs, ys, cs

    def close(self):
        self.fine.close()
        self.coarse.close()


def he_init(seed: int = 0):
    """Initial parameters (W ~ N(0, 2 / fan_in), last layer x 0.1, zero biases),
    laid out as W1[32][25] b1 W2[32][32] b2 W3[32][32] b3 w4[32] b4."""
    import torch
    g = torch.Generator().manual_seed(seed)
    parts = []
    for rows, cols, scale in ((32, NFEAT, 1.0), (32, 32, 1.0), (32, 32, 1.0), (1, 32, 0.1)):
        parts.append(torch.randn(rows * cols, generator=g) * math.sqrt(2.0 / cols) * scale)
        parts.append(torch.zeros(rows))
    w = torch.cat(parts)
    assert w.numel() == V.VP_NET_NPARAM
    return w.cuda()


def train_net(X, y, iters: int = 1500, batch: int = 32768, lr: float = 2e-3, seed: int = 0, stream=None,
              w0=None, coef=None):
    """Adam over minibatches; returns (weights, losses).  With coef the rows
    are cell pairs (2m, 2m + 1) and the loss is the mean squared cell-update
    residual sum_k coef_k (g_k - y_k); without, the mean squared error.
    w0: initial parameters (VP_NET_NPARAM floats, e.g. a He initialisation).
    Everything runs on the current torch stream (the minibatch gathers and
    the library's kernels must be ordered); `stream` is accepted for symmetry
    and waited on first."""
    import torch
    cur = torch.cuda.current_stream()
    if stream is not None and hasattr(stream, "cuda_stream"):
        cur.wait_stream(stream)
    stream = cur
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    w = (w0 if w0 is not None else he_init(seed)).clone().float().cuda()
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    grad = torch.zeros_like(w)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    group = 1 if coef is None else 2
    n = y.numel() // group
    hist = []
    for it in range(1, iters + 1):
        idx = torch.randint(0, n, (min(batch // group, n),), device="cuda", generator=g)
        if group == 2:
            idx = torch.stack([2 * idx, 2 * idx + 1], dim=1).reshape(-1)
        Xb = X[idx].contiguous()
        yb = y[idx].contiguous()
        cb = coef[idx].contiguous() if coef is not None else None
        loss.zero_()
        V.vp_net_grad(Xb, yb, yb.numel(), w, grad, loss, stream, coef=cb, group=group)
        V.vp_net_adam(w, m, v, grad, it, lr * (0.1 ** (it / iters)), stream)
        if it % 50 == 0 or it == iters:
            hist.append(float(loss.item()))
    return w, hist


def heldout_loss(w, X, y, coef) -> float:
    """Mean squared cell-update residual of the network w over the pairs
    (X, y, coef), computed by the training kernel on the current stream."""
    import torch
    grad = torch.zeros_like(w)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    V.vp_net_grad(X, y, y.numel(), w, grad, loss, torch.cuda.current_stream(), coef=coef, group=2)
    return float(loss.item())


def train_select(X, y, coef, seeds=(0, 1, 2), holdout: float = 0.05, split_seed: int = 12345, **kw):
    """Train one network per seed on the cell pairs outside a random held-out
    fraction and keep the one with the lowest held-out loss (the spread
    between initialisations is as large as the gain of a better input set).
    Returns (weights, loss history of the kept run, held-out loss per seed)."""
    import torch
    n = y.numel() // 2
    g = torch.Generator(device="cuda")
    g.manual_seed(split_seed)
    perm = torch.randperm(n, device="cuda", generator=g)
    nh = max(1, int(n * holdout))

    def rows(p):
        return torch.stack([2 * p, 2 * p + 1], dim=1).reshape(-1)

    ti, hi = rows(perm[nh:]), rows(perm[:nh])
    Xt, yt, ct = X[ti].contiguous(), y[ti].contiguous(), coef[ti].contiguous()
    Xh, yh, ch = X[hi].contiguous(), y[hi].contiguous(), coef[hi].contiguous()
    best, losses = None, []
    for sd in seeds:
        w, hist = train_net(Xt, yt, seed=sd, coef=ct, **kw)
        lh = heldout_loss(w, Xh, yh, ch)
        losses.append(lh)
        if best is None or lh < best[0]:
            best = (lh, w, hist)
    return best[1], best[2], losses


def restricted_initial_state(dims: int, nx: int, nv_fine: int, factor: int, k: float, alpha: float,
                             stream=None):
    """Coarse initial f as the mean of the fine point values (the state the
    training pairs are built on); factor 1 gives the fine state itself."""
    import torch
    fine = V.Simulation(landau_grid(dims, nx, nv_fine, k), precision=V.VP_F32, stream=stream)
    V.vp_init_f(fine.ctx, *_landau_ic(dims, k, alpha))
    fine.sync()
    if factor == 1:
        out = fine.f.clone()
    else:
        NX = nx ** dims
        nc = nv_fine // factor
        out = torch.empty(NX * nc ** dims, dtype=torch.float32, device="cuda")
        if dims == 2:
            V.vp_restrict_velocity(fine.f, out, NX, nv_fine, nv_fine, factor, factor, stream)
        else:
            V.vp_restrict_velocity(fine.f, out, NX, nv_fine, 1, factor, 1, stream)
    fine.sync()
    fine.close()
    return out


def run_sweeps(grid: dict, f0, dt: float, steps: int, wts, use_net: int, stream=None):
    """The KDK run of vp_learned_step issued sweep by sweep (not graphed):
    half kicks, learned drifts (x_D .. x_1) with the given use_net mode,
    field solve, half kicks.  For accuracy comparisons of the modes."""
    sim = V.Simulation(grid, precision=V.VP_F32, stream=stream)
    sim.stream.wait_stream(sim.torch.cuda.current_stream())
    with sim.torch.cuda.stream(sim.stream):
        sim.f.copy_(f0.to(sim.f.dtype))
    sim.field()
    D = grid["dims"]
    for _ in range(steps):
        for d in range(D):
            V.vp_kick_sweep(sim.ctx, d, 0.5 * dt, sim.accel[d * sim.NX:])
        for d in reversed(range(D)):
            V.vp_learned_sweep(sim.ctx, 0, d, dt, None, wts, use_net)
        sim.field()
        for d in range(D):
            V.vp_kick_sweep(sim.ctx, d, 0.5 * dt, sim.accel[d * sim.NX:])
    sim.sync()
    return sim


def run(grid: dict, f0, dt: float, steps: int, wts=None, stream=None, precision: int = V.VP_F32):
    """KDK run on `grid` from the state f0 with plain sweeps (vp_step), or
    with learned spatial sweeps when wts is given (vp_learned_step); both
    replay the step as a CUDA graph.  Returns the Simulation (caller closes)."""
    sim = V.Simulation(grid, precision=precision, stream=stream)
    # f0 may still be in flight on the caller's stream
    sim.stream.wait_stream(sim.torch.cuda.current_stream())
    with sim.torch.cuda.stream(sim.stream):
        sim.f.copy_(f0.to(sim.f.dtype))
    sim.field()
    if steps > 0:
        if wts is None:
            sim.step(dt, steps, split=V.VP_SPLIT_KDK)
        else:
            sim.learned_step(dt, steps, wts, split=V.VP_SPLIT_KDK)
    sim.sync()
    return sim
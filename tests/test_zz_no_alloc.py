"""The allocation-free periodic Poisson entry point (vp_poisson_periodic_noalloc).

Some callers cannot allocate device memory while they run (their memory is
owned and budgeted by their own pool, or they cannot afford the device-wide
synchronisation of cudaMalloc/cudaFree).  The entry point keeps its FFT work
array in a static device array instead.  This test calls it through the C ABI
twice in a row (the second call reuses the array the first one left behind)
and checks each result against the context-based solver vp_poisson_solve.
It is collected last so that a failure here cannot hide an earlier one, and
it passes both alone in a fresh process and after the other tests.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_1702_08521_gb300 import vlasov as V

pytestmark = pytest.mark.gpu

GRIDS = [
    dict(dims=2, nx=[48, 40], nv=[2, 2], xlo=[0.0, 0.0], xhi=[4 * math.pi, 3.0], vlo=[-1.0, -1.0],
         vhi=[1.0, 1.0], pois_order=6, coupling=-1.0, rho_bg=1.0),
    dict(dims=1, nx=[256], nv=[2], xlo=[0.0], xhi=[2.0], vlo=[-1.0], vhi=[1.0], pois_order=4,
         coupling=4 * math.pi, rho_bg=0.0),
    dict(dims=3, nx=[16, 12, 8], nv=[2, 2, 2], xlo=[0.0] * 3, xhi=[1.0, 1.5, 2.0], vlo=[-1.0] * 3,
         vhi=[1.0] * 3, pois_order=2, coupling=-1.0, rho_bg=1.0),
]


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


@pytest.mark.parametrize("spec", GRIDS)
def test_noalloc_matches_context_solver_twice(spec):
    import torch
    g = V.make_grid(**spec, precision=V.VP_F64)
    stream = torch.cuda.Stream()
    ctx = V.vp_create(g, stream)
    NX = int(np.prod(spec["nx"]))
    D = spec["dims"]
    rng = np.random.default_rng(NX)
    try:
        for call in range(2):
            rho = torch.as_tensor(1.0 + 0.3 * rng.standard_normal(NX), device="cuda")
            phi_ref = torch.zeros(NX, dtype=torch.float64, device="cuda")
            acc_ref = torch.zeros(D * NX, dtype=torch.float64, device="cuda")
            phi_new = torch.full((NX,), float("nan"), dtype=torch.float64, device="cuda")
            acc_new = torch.full((D * NX,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            V.vp_poisson_solve(ctx, rho, phi_ref, acc_ref)
            rc = V.vp_poisson_periodic_noalloc(g, stream, rho, phi_new, acc_new)
            assert rc == V.VP_OK, (call, rc)
            stream.synchronize()
            assert _rel(phi_new, phi_ref) <= 1e-12, call
            assert _rel(acc_new, acc_ref) <= 1e-12, call
    finally:
        V.vp_destroy(ctx)


def test_noalloc_rejects_grids_beyond_its_limit():
    import torch
    big = V.make_grid(dims=2, nx=[1024, 512], nv=[1, 1], xlo=[0, 0], xhi=[1, 1], vlo=[-1, -1],
                      vhi=[1, 1], precision=V.VP_F64)
    rho = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert V.vp_poisson_periodic_noalloc(big, None, rho, None, rho) == V.VP_EINVAL
    iso = V.make_grid(dims=3, nx=[4, 4, 4], nv=[1, 1, 1], xlo=[0] * 3, xhi=[1] * 3, vlo=[-1] * 3,
                      vhi=[1] * 3, poisson=V.VP_POIS_ISOLATED)
    assert V.vp_poisson_periodic_noalloc(iso, None, rho, None, rho) == V.VP_EINVAL

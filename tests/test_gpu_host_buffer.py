"""vp_host_alloc / vp_host_free: page-locked host buffers on transparent huge
pages for the copies of f (through the C ABI): zero filled, exact round trips
through vp_upload_f / vp_download_f, a buffer of several huge pages, and the
argument checks."""
import ctypes

import numpy as np
import pytest

from paper_1702_08521_gb300 import vlasov as V

pytestmark = pytest.mark.gpu


def test_host_buffer_round_trip():
    g = dict(dims=1, nx=[64], nv=[96], xlo=[0.0], xhi=[1.0], vlo=[-3.0], vhi=[3.0])
    sim = V.Simulation(g, precision=V.VP_F32)
    n = V.vp_num_cells(sim.ctx)
    buf = V.HostBuffer(n * 4)
    a = buf.array(np.float32)
    assert a.size == n and not a.any()
    a[:] = np.random.default_rng(3).random(n, dtype=np.float32)
    V.vp_upload_f(sim.ctx, buf, n * 4)
    sim.sync()
    assert np.array_equal(sim.f.cpu().numpy(), a)
    want = 2.0 * a
    sim.f.mul_(2.0)
    import torch
    torch.cuda.synchronize()
    V.vp_download_f(sim.ctx, buf, n * 4)
    sim.sync()
    assert np.array_equal(buf.array(np.float32), want)
    buf.close()
    buf.close()  # a second close does nothing
    sim.close()


def test_host_buffer_of_several_huge_pages_and_argument_checks():
    nbytes = (3 << 29) + 12345  # 1.5 GB and a ragged tail: several huge pages of any size in use
    buf = V.HostBuffer(nbytes)
    arr = buf.array(np.uint8)
    assert arr.size == nbytes
    arr[::1 << 20] = 7
    arr[-1] = 9
    assert int(arr[::1 << 20].sum()) == 7 * len(range(0, nbytes, 1 << 20)) + (9 - 7 if (nbytes - 1) % (1 << 20) == 0 else 0)
    assert arr[-1] == 9
    buf.close()
    lib = V.load()
    p = ctypes.c_void_p()
    assert lib.vp_host_alloc(0, ctypes.byref(p)) == V.VP_EINVAL
    assert lib.vp_host_alloc(64, None) == V.VP_EINVAL
    assert lib.vp_host_free(ctypes.c_void_p(4096)) == V.VP_EINVAL

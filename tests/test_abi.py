"""The C-ABI library builds, loads and exports every function that
include/vlasov.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

from paper_1702_08521_gb300 import _build, vlasov

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(vp_\w+)\s*\(", src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    try:
        path = _build.build()
    except RuntimeError as e:  # pragma: no cover
        pytest.fail(f"library build failed: {e}")
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("vp_create", "vp_bind_f", "vp_init_f", "vp_drift_sweep", "vp_kick_sweep",
                     "vp_density_moment", "vp_poisson_solve", "vp_diagnostics", "vp_step",
                     "vp_last_error", "vp_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_reports_bad_grid_without_gpu_work(lib):
    vlasov.load()
    g = vlasov.make_grid(1, [8], [8], [0.0], [1.0], [-1.0], [1.0], order=6)
    with pytest.raises(vlasov.VpError):
        vlasov.vp_create(g)


def test_null_context_is_rejected(lib):
    L = vlasov.load()
    assert L.vp_drift_sweep(None, 0, 0.1) == vlasov.VP_EINVAL
    assert L.vp_last_error(None) == b"null context"
    assert L.vp_num_cells(None) == 0

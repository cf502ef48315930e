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


def header_defines():
    """#define VP_<NAME> <integer> of include/vlasov.h."""
    src = open(os.path.join(ROOT, "include", "vlasov.h")).read()
    out = {}
    for m in re.finditer(r"^#define\s+(VP_\w+)\s+\(?(-?\d+)\)?", src, flags=re.M):
        out[m.group(1)] = int(m.group(2))
    return out


def test_binding_constants_match_the_header():
    """Every integer constant the binding defines under a header name has the
    header's value (error codes, schemes, boundary and initial-condition kinds)."""
    hdr = header_defines()
    shared = [n for n in hdr if hasattr(vlasov, n)]
    assert len(shared) >= 20, shared
    for n in shared:
        assert getattr(vlasov, n) == hdr[n], n
    for n in ("VP_ECFL", "VP_SCHEME_SL", "VP_SCHEME_RK", "VP_IC_SPHERE", "VP_NET_NPARAM"):
        assert n in hdr and hasattr(vlasov, n), n


def test_grid_struct_matches_the_header():
    """The ctypes vp_grid lists the header struct's fields in order."""
    src = open(os.path.join(ROOT, "include", "vlasov.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} vp_grid;", src, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(None, 1)[1].split(","):
            names.append(re.sub(r"\[.*\]", "", part).strip())
    assert [f[0] for f in vlasov.vp_grid._fields_] == names


def test_host_buffer_and_ensemble_calls_check_their_arguments_without_gpu_work(lib):
    """Argument checks that return before any CUDA call: a zero-byte or
    output-less host allocation, freeing a pointer the library did not hand
    out, and the ensemble's flat-vote calls on a null ensemble."""
    L = vlasov.load()
    p = ctypes.c_void_p()
    assert L.vp_host_alloc(0, ctypes.byref(p)) == vlasov.VP_EINVAL
    assert p.value is None
    assert L.vp_host_alloc(64, None) == vlasov.VP_EINVAL
    assert L.vp_host_free(ctypes.c_void_p(4096)) == vlasov.VP_EINVAL
    assert L.vp_host_free(None) == vlasov.VP_EINVAL
    on = ctypes.c_int(7)
    assert L.vp_ensemble_set_flat_vote(None, 1) == vlasov.VP_EINVAL
    assert L.vp_ensemble_get_flat_vote(None, ctypes.byref(on)) == vlasov.VP_EINVAL
    assert on.value == 7

"""The C-ABI library builds, loads and exports every symbol include/aao.h declares;
argument validation that needs no GPU (no compute call is made here)."""
import ctypes

import pytest

import paper_2306_03574_gb300 as aao


@pytest.fixture(scope="module")
def L():
    from paper_2306_03574_gb300 import build
    build.build()
    return aao.lib()


def test_every_header_symbol_exported(L):
    names = aao.header_functions()
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(L):
    assert aao.aao_status_str(aao.AAO_OK) == "AAO_OK"
    assert aao.aao_status_str(aao.AAO_ESINGULAR) == "AAO_ESINGULAR"
    assert aao.aao_status_str(aao.AAO_ETIMEOUT) == "AAO_ETIMEOUT"
    assert aao.aao_status_str(99) == "AAO_UNKNOWN"


@pytest.mark.parametrize("kw,status", [
    (dict(dim=0), aao.AAO_EINVAL),
    (dict(dim=4), aao.AAO_EINVAL),
    (dict(alpha=0.0), aao.AAO_EINVAL),
    (dict(alpha=1.5), aao.AAO_EINVAL),
    (dict(tau=0.0), aao.AAO_EINVAL),
    (dict(tau=float("nan")), aao.AAO_EINVAL),
    (dict(c2=-1.0), aao.AAO_EINVAL),
    (dict(scheme=3), aao.AAO_EINVAL),
    (dict(nt=1), aao.AAO_EINVAL),
    (dict(N=100), aao.AAO_EUNSUPPORTED),
    (dict(N=31), aao.AAO_EUNSUPPORTED),
    (dict(N=1023), aao.AAO_EUNSUPPORTED),
    (dict(nt=96), aao.AAO_EUNSUPPORTED),
    (dict(nt=2048), aao.AAO_EUNSUPPORTED),
    (dict(precision=7), aao.AAO_EINVAL),
])
def test_create_rejects_bad_arguments(L, kw, status):
    args = dict(dim=2, N=63, nt=64, tau=1 / 64, alpha=1e-2, c2=1.0, precision=0, nrhs_max=1, scheme=0)
    args.setdefault("variable_coefficient", False)
    args.update(kw)
    st, h = aao.aao_create(raw_status=True, **args)
    assert st == status, (st, aao.aao_last_error())
    assert h is None
    assert aao.aao_last_error() != ""


def test_null_pointers_rejected(L):
    h = ctypes.c_void_p()
    assert L.aao_create(None, 64, 1 / 64, 0.1, 0, None, ctypes.byref(h)) == aao.AAO_EINVAL
    assert L.aao_destroy(None) == aao.AAO_OK
    assert L.aao_workspace_bytes(None) == 0
    assert L.aao_launch_count(None) == 0
    assert L.aao_apply_prec(None, None, None, 1, None) == aao.AAO_EINVAL
    assert L.aao_minres_solve(None, None, None, 0, 1, 1e-8, 10, None, None) == aao.AAO_EINVAL
    assert L.aao_autotune(None, None, None) == aao.AAO_EINVAL
    assert L.aao_set_coefficient(None, None, None) == aao.AAO_EINVAL


def test_serve_argument_validation(L):
    """Serving entry points reject bad arguments before touching the GPU."""
    st, srv = aao.aao_serve_create(0, 4, raw_status=True)
    assert st == aao.AAO_EINVAL and srv is None
    st, srv = aao.aao_serve_create(1 << 30, 0, raw_status=True)
    assert st == aao.AAO_EINVAL
    st, srv = aao.aao_serve_create(1 << 30, 65, raw_status=True)
    assert st == aao.AAO_EINVAL
    assert L.aao_serve_submit(None, None, None) == aao.AAO_EINVAL
    assert L.aao_serve_poll(None, 1, None) == aao.AAO_EINVAL
    assert L.aao_serve_destroy(None) == aao.AAO_OK

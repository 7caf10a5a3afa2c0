"""The C ABI library builds, loads and exports every entry point declared in include/*.h.
Host-side argument validation is exercised without touching a GPU."""
import ctypes as C
import glob
import os
import re

import pytest

from paper_2303_15861_gb300 import adr, build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    path = build_lib.build()
    return adr.load_library(path)


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(adr_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = _declared_functions()
    for required in ("adr_create", "adr_set_coeffs", "adr_step", "adr_integrate", "adr_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def _params(**kw):
    p = adr.adr_params()
    p.dim = kw.get("dim", 3)
    for i, n in enumerate(kw.get("n", (8, 8, 8))):
        p.n[i] = n
    p.tau = kw.get("tau", 1e-3)
    p.scheme = kw.get("scheme", 0)
    p.precision = kw.get("precision", 0)
    return p


@pytest.mark.parametrize("kw,status", [
    (dict(dim=4), 1),
    (dict(n=(1, 8, 8)), 1),
    (dict(tau=0.0), 1),
    (dict(tau=-1.0), 1),
    (dict(scheme=7), 1),
    (dict(precision=9), 1),
    (dict(precision=2), 8),
])
def test_create_rejects_invalid_params_on_host(lib, kw, status):
    """Invalid parameters are refused before any CUDA call; the message is kept."""
    ctx = C.c_void_p()
    p = _params(**kw)
    assert lib.adr_create(C.byref(p), None, C.byref(ctx)) == status
    assert not ctx.value
    assert len(lib.adr_last_error(None)) > 0


def test_null_arguments(lib):
    assert lib.adr_create(None, None, None) == 1
    assert lib.adr_kernels_per_step(None) == -1
    lib.adr_destroy(None)

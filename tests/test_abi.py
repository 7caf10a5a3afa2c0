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
    (dict(scheme=42), 1),
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


def _batch_params(sizes, **kw):
    p = _params(dim=kw.get("dim", 2), n=(0, 0, 0), scheme=kw.get("scheme", 1), precision=kw.get("precision", 1))
    flat = [v for d in sizes for v in d]
    arr = (C.c_int * max(1, len(flat)))(*flat)
    p.batch = kw.get("batch", len(sizes))
    p.n_batch = C.cast(arr, C.POINTER(C.c_int)) if kw.get("with_sizes", True) else None
    p.batch_tile = kw.get("batch_tile", 0)
    return p, arr


@pytest.mark.parametrize("kw,status", [
    (dict(dim=3), 1),                       # batched contexts are 2-D
    (dict(with_sizes=False), 1),            # n_batch missing
    (dict(batch=-1), 1),
    (dict(precision=3, sizes=[(48, 48), (257, 64)]), 1),   # mixed batches: instances up to 256 per direction
    (dict(precision=2), 8),                 # TF32x3 is not built
    (dict(batch_tile=48), 1),
    (dict(sizes=[(48, 48), (1, 64)]), 1),   # an instance below the minimum size
])
def test_create_batch_rejects_invalid_params_on_host(lib, kw, status):
    """Batched contexts validate their parameters before any CUDA call."""
    sizes = kw.pop("sizes", [(48, 48), (64, 32)])
    p, keep = _batch_params(sizes, **kw)
    ctx = C.c_void_p()
    assert lib.adr_create(C.byref(p), None, C.byref(ctx)) == status
    assert not ctx.value
    assert len(lib.adr_last_error(None)) > 0
    del keep


def test_batch_plan_needs_a_context(lib):
    assert lib.adr_get_batch_plan(None, 1, None, None) == 1
    assert lib.adr_get_instance_info(None, 0, None, None, None) == 1


def _periodic_params(**kw):
    p = _params(dim=kw.get("dim", 2), n=kw.get("n", (16, 16, 1)), precision=kw.get("precision", 0),
                scheme=kw.get("scheme", 6))
    p.periodic = kw.get("periodic", 1)
    p.length = kw.get("length", 1.0)
    p.phi_route = kw.get("phi_route", 0)
    p.bc_hi = kw.get("bc_hi", 0)
    p.form = kw.get("form", 0)
    p.batch = kw.get("batch", 0)
    return p


@pytest.mark.parametrize("kw,status", [
    (dict(n=(12, 16, 1)), 1),          # not a power of two
    (dict(n=(8192, 16, 1)), 1),        # x1 lines beyond 4096 points
    (dict(n=(16, 2048, 1)), 1),        # other lines beyond 1024 points
    (dict(form=2), 1),
    (dict(n=(1, 16, 1)), 1),
    (dict(length=0.0), 1),
    (dict(length=float("inf")), 1),
    (dict(precision=3), 8),            # the Fourier path runs in FP64 or FP32
    (dict(phi_route=1), 1),
    (dict(bc_hi=1, form=1), 1),
    (dict(periodic=2), 1),
    (dict(batch=2), 8),
    (dict(scheme=42), 1),
])
def test_create_rejects_invalid_periodic_params_on_host(lib, kw, status):
    ctx = C.c_void_p()
    p = _periodic_params(**kw)
    assert lib.adr_create(C.byref(p), None, C.byref(ctx)) == status
    assert not ctx.value
    assert len(lib.adr_last_error(None)) > 0


def test_periodic_entry_points_reject_null_contexts(lib):
    dp = C.POINTER(C.c_double)
    assert lib.adr_set_coeffs_periodic(None, dp(), dp(), dp()) == 1


def test_measure_peak_validates_arguments_on_host(lib):
    out = C.c_double()
    assert lib.adr_measure_peak(0, 16, None) == 1
    assert lib.adr_measure_peak(7, 16, C.byref(out)) == 1
    assert lib.adr_measure_peak(0, 0, C.byref(out)) == 1
    assert lib.adr_measure_peak(1, (1 << 20) + 1, C.byref(out)) == 1


def test_bounded_wait_probe_validates_arguments_on_host(lib):
    assert lib.adr_test_bounded_wait(None, 1.0) == 1


def test_factor_slice_query_validates_arguments_on_host(lib):
    n = C.c_int(-1)
    assert lib.adr_tc_factor_slices(None, C.byref(n)) == 1
    assert lib.adr_tc_factor_slices(None, None) == 1

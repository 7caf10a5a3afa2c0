"""Table 1 through the library's host code (adr_stability_bound: bisection on the stability
functions of Theorems 2.1-2.7), against the values the paper prints. Lawson4 has no printed
bound; the library's is checked against a bisection over the oracle's own Lawson4 step on
the scalar test equation. Host arithmetic only: no GPU is needed."""
import json
import os

import numpy as np
import pytest

from oracle import adr_oracle as O
from paper_2303_15861_gb300 import adr, build_lib

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def lib():
    return adr.load_library(build_lib.build())


def test_library_bounds_match_table1(lib):
    with open(os.path.join(GOLDEN, "table1_stability_bounds.json")) as f:
        gold = json.load(f)
    for scheme, ref in gold["bounds"].items():
        assert abs(adr.adr_stability_bound(scheme) - ref) <= gold["tolerance"], scheme


def test_lawson4_bound_matches_the_oracle_stepper(lib):
    z = -np.concatenate([np.logspace(-4, 9, 20001), np.linspace(0.0, 50.0, 20001)])

    def stable(lam):
        ops = O.ScalarOps(lam * z, lambda u: (1.0 - lam) * z * u, 1.0)
        return np.all(np.abs(O.SCHEMES["lawson4"](ops, np.ones_like(z))) <= 1 + 1e-12)

    lo, hi = 0.0, 1.0
    for _ in range(30):
        mid = 0.5 * (lo + hi)
        lo, hi = (lo, mid) if stable(mid) else (mid, hi)
    assert abs(adr.adr_stability_bound("lawson4") - hi) <= 1e-3


def test_stability_bound_rejects_unknown_schemes(lib):
    import ctypes as C
    out = C.c_double()
    assert lib.adr_stability_bound(42, C.byref(out)) == 1
    assert lib.adr_stability_bound(0, None) == 1

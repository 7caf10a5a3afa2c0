"""Element-wise parity checks shared by the GPU tests.

Every comparison of a GPU result with its reference asserts three things:
  * the relative l2 error over all nodes (the parity measure of the workloads);
  * the relative maximum norm max|got - ref| / max|ref|, the norm the paper's Section 5
    reports, which no single bad tile, ragged tail or face row can hide under;
  * each boundary-adjacent plane (first and last index along every axis) on its own scale:
    the l2 error of the plane against the plane's own norm. Near Dirichlet faces the
    solution is small, so a wrong ghost value or face coefficient is an O(1) error of that
    plane even where it is negligible against the whole array. A plane on which the solution
    all but vanishes (a periodic problem whose solution is localised away from the box edge)
    is measured against a floor instead: 1e-3 of the norm a plane would have if the array's
    norm were spread evenly over its entries.
The max-norm bound defaults to 4x the l2 bound (the GPU runs measure at most 1.3x); a face
bound defaults to 1000x the l2 bound: a precision whose error is a fixed fraction of the
array's maximum (the fixed-point slices of the mixed path) shows up larger on a plane whose
values are ~h of the maximum, by up to 2e3 on the 256^3 workload.
Set PARITY_LOG to a file path to append every measured triple (for choosing bounds).
"""
import json
import os

import numpy as np

from oracle import adr_oracle as O


def boundary_planes(a):
    """(axis, side, plane) for the first and last plane along every axis of a."""
    for ax in range(a.ndim):
        if a.shape[ax] < 2:
            continue
        yield ax, 0, np.take(a, 0, axis=ax)
        yield ax, -1, np.take(a, -1, axis=ax)


FACE_FLOOR = 1e-3


def face_errors(got, ref):
    """Largest l2 error of a boundary-adjacent plane relative to the plane's own norm (or to the
    floor, for planes on which the solution all but vanishes)."""
    worst = 0.0
    total = float(np.linalg.norm(ref))
    for (ax, side, g), (_, _, r) in zip(boundary_planes(got), boundary_planes(ref)):
        even = total * np.sqrt(r.size / ref.size)
        scale = max(float(np.linalg.norm(r)), FACE_FLOOR * even)
        e = float(np.linalg.norm(g - r))
        if scale == 0.0:
            worst = max(worst, 0.0 if e == 0.0 else np.inf)
        else:
            worst = max(worst, e / scale)
    return worst


def assert_parity(got, ref, l2, inf=None, face=None, what=""):
    """Assert relative l2 < l2, relative max norm < inf (default 4 l2) and, for arrays of two
    or more dimensions, every boundary-adjacent plane within face (default 1000 l2) of its own
    norm (face=False skips the planes). Returns (rel_l2, rel_inf, worst plane)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    assert np.isfinite(got).all(), f"{what}: non-finite values in the result"
    inf = 4.0 * l2 if inf is None else inf
    e2, ei = O.rel_l2(got, ref), O.rel_inf(got, ref)
    ef = face_errors(got, ref) if (face is not False and got.ndim >= 2) else 0.0
    log = os.environ.get("PARITY_LOG")
    if log:
        with open(log, "a") as f:
            f.write(json.dumps({"what": str(what), "shape": list(got.shape), "l2": e2, "inf": ei, "face": ef,
                                "tol_l2": l2, "tol_inf": inf}) + "\n")
    assert e2 < l2, f"{what}: relative l2 {e2:.3e} >= {l2:.1e} (max norm {ei:.3e})"
    assert ei < inf, f"{what}: relative max norm {ei:.3e} >= {inf:.1e} (l2 {e2:.3e})"
    if face is not False and got.ndim >= 2:
        ft = 1000.0 * l2 if face is None else face
        assert ef < ft, f"{what}: a boundary-adjacent plane is off by {ef:.3e} of its own norm (bound {ft:.1e})"
    return e2, ei, ef

"""The oracle against numbers the paper prints for its experiments.

The three-dimensional experiment (Section 5.2, Eq. (adr3d): a Lap u, Dirichlet faces at
x_mu = 0, Neumann faces at x_mu = 1; the figure of errors against lambda, N = 2^4, m = 2^8,
T = 1/4, b = -0.01 and -1; tests/golden/e4_lambda_scan_paper.json): every printed point of the
four schemes matches to 1e-4 relative against a Lawson2b reference with 2^13 steps; asserted
within 1e-3, with the printed argmin.

The one-dimensional linear diffusion problem a(x) u_xx (Section 4, Eq. (adlinearzero); the
figures of errors against the number of steps, one panel per lambda; tests/golden/
e1_errors_paper.json), against the exact semidiscrete solution, for the printed points with
m <= 256 (the figures also hold short segments that run off the plotted range above 1e-1; they
are not data points). Where lambda is at or above the scheme's Table 1 bound (unconditionally
stable) every point matches: to seven digits at lambda = 1 and within 0.2% at the bound;
asserted within 3e-3. Below the bound the errors come from growing modes and amplify rounding
differences: the points agree within 30%, asserted within [0.7, 1.4].

The one-dimensional nonlinear diffusion-reaction problem (Section 4, Eq. (adnonlinear); the
figure of errors against lambda; tests/golden/e2_lambda_errors_paper.json): every printed point
of the eight schemes the paper plots and this project implements matches to 0.1%, against a
Lawson4 reference with 2^14 steps; asserted within 1%.

The lambda scan of the two-dimensional periodic
experiment (Section 5.1, Eq. (ad2d); the errors of the figure of errors against lambda, top panels,
N = 2^6, m = 2^8, T = 4; the chosen lambda of each scheme in the table of lambda values of
Section 5.1). Stored in tests/golden/e3_lambda_scan_paper.json.

The error is the paper's: the infinity norm at T relative to a reference integrated by Lawson2b
with a small step (opening of Section 5); here 2^13 steps.

At N = 2^8 (the bottom panels) every scheme, Lawson2a included, matches the printed errors within
0.2% at the endpoints of each curve (asserted within 3e-3). At N = 2^6 (the top panels):

Readings and tolerances. Over every printed point of five schemes (stabilized Lawson-Euler,
Lawson-Euler, exponential Euler, stabilized Lawson2, erk2p1) the oracle's error is 0.979 to 1.013
times the paper's, with the same argmin lambda; the band asserted is [0.97, 1.02]. The remaining
2% offset is common to all five schemes and all lambda, so it is read as a difference in the
normalisation or reference, not in a scheme. Lawson2a's curve deviates more (0.94 to 1.17 of the
paper's, argmin 0.57 against the printed 0.527 on a flat minimum): its band is [0.93, 1.18],
and the deviation is listed as unexplained.
"""
import json
import os

import numpy as np
import pytest

from oracle import adr_oracle as O
from paper_2303_15861_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "e3_lambda_scan_paper.json")


@pytest.fixture(scope="module")
def e3():
    g = json.load(open(GOLDEN))
    w, L, a, b = W.config_e3(n=g["N"], scheme="lawson_euler", m=g["m"], T=g["T"])
    ref = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, g["T"] / 8192, 8192, "lawson2b")
    return g, w, L, a, b, ref


def curve(e3, scheme):
    g, w, L, a, b, ref = e3
    out = []
    for lam, paper in g["points"][scheme]:
        u = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, g["T"] / g["m"], g["m"], scheme, lam=lam)
        out.append((lam, np.abs(u - ref).max() / np.abs(ref).max(), paper))
    return out


@pytest.mark.parametrize("scheme", ["stabilized_lawson_euler", "lawson_euler", "exponential_euler",
                                    "stabilized_lawson2", "erk2p1"])
def test_e3_lambda_scan_errors_and_argmin_match_the_paper(e3, scheme):
    c = curve(e3, scheme)
    for lam, ours, paper in c:
        assert 0.97 <= ours / paper <= 1.02, (scheme, lam, ours, paper)
    assert min(c, key=lambda t: t[1])[0] == min(c, key=lambda t: t[2])[0]


def test_e3_lambda_scan_lawson2a_within_its_documented_band(e3):
    for lam, ours, paper in curve(e3, "lawson2a"):
        assert 0.93 <= ours / paper <= 1.18, (lam, ours, paper)


GOLDEN_E2 = os.path.join(os.path.dirname(__file__), "golden", "e2_lambda_errors_paper.json")


@pytest.fixture(scope="module")
def e2():
    g = json.load(open(GOLDEN_E2))
    w, L, a, b = W.config_e2(n=g["N"], m=g["m"], T=g["T"])
    ref = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, g["T"] / 16384, 16384, "lawson4")
    return g, w, L, a, b, ref


@pytest.mark.parametrize("scheme", ["stabilized_lawson_euler", "lawson_euler", "exponential_euler", "etd2rk",
                                    "stabilized_lawson2", "erk2p1", "lawson2a", "lawson2b"])
def test_e2_errors_match_the_paper(e2, scheme):
    g, w, L, a, b, ref = e2
    for lam, paper in g["points"][scheme]:
        u = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, g["T"] / g["m"], g["m"], scheme, lam=lam)
        ours = np.abs(u - ref).max() / np.abs(ref).max()
        assert abs(ours / paper - 1.0) <= 0.01, (scheme, lam, ours, paper)


GOLDEN_E1 = os.path.join(os.path.dirname(__file__), "golden", "e1_errors_paper.json")


@pytest.fixture(scope="module")
def e1():
    g = json.load(open(GOLDEN_E1))
    w, L, a, b = W.config_e1(n=g["N"], T=g["T"])
    prob = O.PeriodicProblem(w.dims, L, a, b, w.r_poly, form="adelta")
    exact = O.periodic_linear_exact(prob, w.u0, g["T"])
    return g, w, L, a, b, exact


# Table 1 bounds on lambda for unconditional stability (tests/golden/table1_stability_bounds.json)
TABLE1 = {"lawson_euler": 0.2178, "etd2rk": 0.5, "exponential_euler": 0.5, "erk2p1": 1.0 / 3.0,
          "stabilized_lawson_euler": 0.18394, "lawson2a": 0.30056, "lawson2b": 0.30056, "stabilized_lawson2": 0.18203}


@pytest.mark.parametrize("panel", ["1", "1/2", "1/3", "0.301", "0.218", "1/(2e)", "0.183", "0.17"])
def test_e1_errors_match_the_paper(e1, panel):
    g, w, L, a, b, exact = e1
    p = g["panels"][panel]
    checked = 0
    for scheme, pts in p["curves"].items():
        stable = p["lambda"] >= TABLE1[scheme] - 1e-4
        for m, paper in pts:
            if m not in (16, 64, 256) or paper > 0.1:
                continue
            u = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, g["T"] / m, m, scheme, lam=p["lambda"],
                                 form="adelta")
            ours = np.abs(u - exact).max() / np.abs(exact).max()
            if stable:
                assert abs(ours / paper - 1.0) <= 3e-3, (panel, scheme, m, ours, paper)
            else:
                assert 0.7 <= ours / paper <= 1.4, (panel, scheme, m, ours, paper)
            checked += 1
    assert checked > 0


GOLDEN_E4 = os.path.join(os.path.dirname(__file__), "golden", "e4_lambda_scan_paper.json")


@pytest.mark.parametrize("b", ["-0.01", "-1"])
def test_e4_lambda_scan_errors_and_argmin_match_the_paper(b):
    g = json.load(open(GOLDEN_E4))
    w = W.config_e4(n=g["N"], b=float(b), scheme="lawson_euler", m=g["m"], T=g["T"])
    kw = dict(bc="mixed", form="adelta")
    ref = O.solve(w.dims, w.a_nodes, w.b, w.r_poly, w.u0, g["T"] / 8192, 8192, "lawson2b", **kw)
    for scheme, pts in g["points"][b].items():
        errs = []
        for lam, paper in pts:
            u = O.solve(w.dims, w.a_nodes, w.b, w.r_poly, w.u0, g["T"] / g["m"], g["m"], scheme, lam=lam, **kw)
            ours = np.abs(u - ref).max() / np.abs(ref).max()
            assert abs(ours / paper - 1.0) <= 1e-3, (b, scheme, lam, ours, paper)
            errs.append(ours)
        assert pts[int(np.argmin(errs))][0] == min(pts, key=lambda t: t[1])[0]


def test_e3_at_2_to_the_8_modes_matches_the_paper():
    """The bottom panels of the same figure (N = 2^8): lambda = 1 of Lawson-Euler, exponential
    Euler and Lawson2a (every endpoint of all six curves was checked the same way; this keeps the
    CPU suite short). Reference: Lawson4 with 2^9 steps."""
    g = json.load(open(GOLDEN))
    w, L, a, b = W.config_e3(n=256, scheme="lawson_euler", m=g["m"], T=g["T"])
    ref = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, g["T"] / 512, 512, "lawson4")
    for scheme in ("lawson_euler", "exponential_euler", "lawson2a"):
        pts = g["points_n256"][scheme]
        for lam, paper in (pts[-1],):
            u = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, g["T"] / g["m"], g["m"], scheme, lam=lam)
            ours = np.abs(u - ref).max() / np.abs(ref).max()
            assert abs(ours / paper - 1.0) <= 3e-3, (scheme, lam, ours, paper)

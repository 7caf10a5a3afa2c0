"""Edge and degenerate cases of the CUDA path, through the C ABI, against the FP64 oracle or
against what the mathematics fixes exactly.

* A zero state stays exactly zero: r(0) = 0, so F(0) = g(0) = 0 and every stage is zero. On the
  mixed paths this runs the slicing with a zero max-abs scale.
* With a constant coefficient a = a_max and no reaction, g = 0 and the problem is linear:
  Lawson-Euler, ETD2RK, Lawson4, exponential Euler, erk2p1 and the Lawson2 schemes are exact
  for it (the remark after Table 1), so m steps give the semidiscrete solution e^{m tau A} u0,
  which the oracle forms from its own Pade factors of m tau A_mu.
* The smallest grids (2 x 2, 2 x 2 x 2, x1 extents not a multiple of 4) and a batch that mixes
  2 x 2 with 256 x 256 instances.
* m = 0 leaves the state untouched.
"""
import dataclasses

import numpy as np
import pytest

from oracle import adr_oracle as O
from paper_2303_15861_gb300 import workloads as W
from parity import assert_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2303_15861_gb300 import adr, build_lib  # noqa: E402

build_lib.build()
adr.load_library()

DT = {"fp64": torch.float64, "fp32": torch.float32, "bf16x3": torch.float32}


def grid_context(dims, tau, scheme, prec, a, b, r):
    c = adr.Context(dims, tau, scheme, prec)
    c.set_coeffs(a, b, r)
    return c


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3"])
@pytest.mark.parametrize("scheme", ["lawson4", "etd2rk", "lawson2a"])
def test_zero_state_stays_zero(prec, scheme):
    dims = (40, 24, 36)
    a, b, r = W.sine_product_coefficient(dims), (10.0, -5.0, 3.0), W.REACTION_U2_1MU
    ctx = grid_context(dims, 2e-3, scheme, prec, a, b, r)
    u = torch.zeros(dims[::-1], dtype=DT[prec], device="cuda")
    ctx.integrate(u, 0.0, 6 * 2e-3, 6)
    ctx.synchronize()
    assert torch.all(u == 0), (scheme, prec)


def small_advection(ws):
    """The instances with b scaled to cell Peclet numbers below one on their grid (a 2 x 2 grid
    has h = 1/3: the drawn b up to 20 would leave A_mu without a real eigenbasis, which the
    library refuses for the phi schemes)."""
    out = []
    for w in ws:
        h = 1.0 / (min(w.dims) + 1)
        bmax = 0.5 * 2.0 * float(np.min(w.a_nodes)) / h       # half the Peclet limit with the smallest a
        scale = min(1.0, bmax / max(1e-30, max(abs(v) for v in w.b)))
        out.append(dataclasses.replace(w, b=tuple(v * scale for v in w.b)))
    return out


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("scheme", ["etd2rk", "lawson4"])
def test_zero_state_stays_zero_batched(prec, scheme):
    ws = small_advection(W.batch_instances([(48, 48), (33, 70), (2, 2)], scheme=scheme))
    ctx = adr.Context(None, ws[0].tau, scheme, prec, batch_dims=[w.dims for w in ws])
    for i, w in enumerate(ws):
        ctx.set_coeffs(w.a_nodes, w.b, w.r_poly, instance=i)
    u = torch.zeros(sum(w.dof for w in ws), dtype=torch.float32, device="cuda")
    ctx.integrate(u, 0.0, 4 * ws[0].tau, 4)
    ctx.synchronize()
    assert torch.all(u == 0)


LINEAR_SCHEMES = ["lawson_euler", "etd2rk", "lawson4", "exponential_euler", "erk2p1", "lawson2a", "lawson2b"]


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("scheme", LINEAR_SCHEMES)
def test_linear_problem_gives_the_exact_semidiscrete_solution(scheme, prec):
    # FP64 1e-12; mixed: 2e-6 for the exponential-only schemes, and for the phi schemes the
    # eigen-route bound of the mixed integration tests (the slices of V_mu and V_mu^-1 are fixed
    # point per row while their entries span kappa(V_mu))
    tol = 1e-12 if prec == "fp64" else (3e-5 if scheme in ("etd2rk", "exponential_euler", "erk2p1") else 2e-6)
    dims = (48, 40, 36)
    amax = 1.3
    a = np.full(tuple(n + 2 for n in dims[::-1]), amax)     # a = a_max: g = (b - beta) . grad u + r = 0
    b, r = (8.0, -6.0, 4.0), (0.0, 0.0, 0.0, 0.0)
    tau, m = 2.5e-3, 8
    u0 = W.smooth_initial_state(dims, noise=1e-3)
    ctx = grid_context(dims, tau, scheme, prec, a, b, r)
    u = torch.tensor(u0, dtype=DT[prec], device="cuda")
    ctx.integrate(u, 0.0, m * tau, m)
    ctx.synchronize()
    prob = O.ADRProblem(dims, a, b, r)
    exact = O.MatrixFunctions(prob, m * tau).exp_action(1.0, u0)
    assert_parity(u.double().cpu().numpy(), exact, tol, what=f"linear {scheme} {prec}")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5), ("bf16x3", 2e-5)])
@pytest.mark.parametrize("dims", [(2, 2), (2, 2, 2), (3, 5), (5, 3, 2), (7, 2, 3)])
@pytest.mark.parametrize("scheme", ["lawson4", "etd2rk"])
def test_smallest_grids_match_oracle(dims, scheme, prec, tol):
    a = W.sine_product_coefficient(dims)
    b, r = (4.0, -3.0, 2.0)[: len(dims)], W.REACTION_U2_1MU
    bb = tuple(b) + (0.0,) * (3 - len(b))
    u0 = 0.5 + 0.1 * np.random.default_rng(3).standard_normal(tuple(dims[::-1]))
    tau, m = 1e-3, 4
    ctx = grid_context(dims, tau, scheme, prec, a, bb, r)
    u = torch.tensor(u0, dtype=DT[prec], device="cuda")
    uin = u.double().cpu().numpy()                   # the state the GPU starts from (FP32-rounded)
    ctx.integrate(u, 0.0, m * tau, m)
    ctx.synchronize()
    ref = O.solve(dims, a, bb, r, uin, tau, m, scheme)
    assert_parity(u.double().cpu().numpy(), ref, tol, what=f"{dims} {scheme} {prec}")


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16x3", 1e-5)])
def test_batch_of_extreme_sizes_matches_oracle(prec, tol):
    """A batch holding the smallest (2 x 2, 2 x 3) and the largest (256 x 256) instances of the
    mixed path, and a long thin one, with ETD2RK over 6 steps."""
    ws = small_advection(W.batch_instances([(2, 2), (256, 256), (2, 3), (250, 7)], scheme="etd2rk"))
    ctx = adr.Context(None, ws[0].tau, "etd2rk", prec, batch_dims=[w.dims for w in ws], kappa_tol=1.0)
    for i, w in enumerate(ws):
        ctx.set_coeffs(w.a_nodes, w.b, w.r_poly, instance=i)
    flat = np.concatenate([w.u0.ravel() for w in ws])
    u = torch.tensor(flat, dtype=torch.float32, device="cuda")
    m = 6
    ctx.integrate(u, 0.0, m * ws[0].tau, m)
    ctx.synchronize()
    h, o = u.double().cpu().numpy(), 0
    for w in ws:
        got = h[o:o + w.dof].reshape(w.dims[::-1])
        o += w.dof
        u0 = np.asarray(w.u0, dtype=np.float32).astype(np.float64)
        ref = O.solve(w.dims, w.a_nodes, w.b, w.r_poly, u0, w.tau, m, "etd2rk")
        assert_parity(got, ref, tol, what=(w.name, prec))


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_zero_steps_leave_the_state_untouched(prec):
    dims = (32, 24, 20)
    a, b, r = W.sine_product_coefficient(dims), (10.0, 10.0, 10.0), W.REACTION_U2_1MU
    ctx = grid_context(dims, 1e-3, "lawson4", prec, a, b, r)
    u = torch.tensor(W.smooth_initial_state(dims), dtype=DT[prec], device="cuda")
    before = u.clone()
    ctx.integrate(u, 0.0, 0.0, 0)
    ctx.synchronize()
    assert torch.equal(u, before)

"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 paths 1e-12 relative l2 (the FP64 requirement of the workloads);
FP32 paths are bounded by FP32 rounding of the stencil and the contractions. Every
comparison is also element by element (tests/parity.py): the relative maximum norm and
each boundary-adjacent plane on its own scale.
Sizes span several CTA tiles and ragged tails; guard bands around every caller-owned
array check that nothing is written out of bounds.
"""
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

GUARD = 1024


def guarded(shape, dtype, fill=None):
    """A device array with NaN guard bands on both sides; returns (full, view)."""
    n = int(np.prod(shape))
    full = torch.full((n + 2 * GUARD,), float("nan"), dtype=dtype, device="cuda")
    view = full[GUARD:GUARD + n].view(shape)
    if fill is not None:
        view.copy_(torch.as_tensor(np.asarray(fill), dtype=dtype))
    return full, view


def check_guards(full):
    g = torch.cat([full[:GUARD], full[-GUARD:]])
    assert torch.isnan(g).all(), "write outside the caller's array"


def make_case(dims, b=None, c=0.5, k=1, noise=1e-3, seed=0):
    b = b if b is not None else (10.0,) * len(dims)
    a = W.sine_product_coefficient(dims, c=c, k=k)
    u0 = W.smooth_initial_state(dims, noise=noise, seed=seed)
    return a, tuple(b) + (0.0,) * (3 - len(b)), W.REACTION_U2_1MU, u0


def context(dims, tau, scheme, prec, a, b, r):
    ctx = adr.Context(dims, tau, scheme, prec)
    ctx.set_coeffs(a, b, r)
    return ctx


DTYPES = {"fp64": torch.float64, "fp32": torch.float32}
# the last two take the TMA-staged 3-D kernel (n1 >= 64, n2 >= 16) with ragged tiles in x1 and
# x2 (tiles of 64 x 16) and a ragged last CTA in x3
STENCIL_DIMS = [(32, 32), (37, 29), (33, 33, 33), (45, 19, 23), (132, 36, 20), (68, 16, 9)]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
@pytest.mark.parametrize("dims", STENCIL_DIMS)
def test_stencil_F_and_g(dims, prec, tol):
    b = (10.0, -7.0, 4.0)[: len(dims)]
    a, bb, r, u0 = make_case(dims, b=b, k=2)
    prob = O.ADRProblem(dims, a, bb, r)
    ctx = context(dims, 1e-3, "lawson4", prec, a, bb, r)
    dt = DTYPES[prec]
    fu, u = guarded(u0.shape, dt, u0)
    fF, F = guarded(u0.shape, dt)
    fg, g = guarded(u0.shape, dt)
    ctx.eval_rhs(u, F, g)
    torch.cuda.synchronize()
    for full in (fu, fF, fg):
        check_guards(full)
    uin = u.double().cpu().numpy()          # the FP32 path sees the rounded state
    refF, refg = prob.F(uin), prob.g(uin)
    assert_parity(F.cpu().numpy(), refF, tol, what=f"F {dims} {prec}")
    assert_parity(g.cpu().numpy(), refg, tol, what=f"g {dims} {prec}")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
@pytest.mark.parametrize("dims", [(32, 32), (70, 45), (33, 33, 33), (45, 19, 23), (130, 65, 67)])
@pytest.mark.parametrize("c", [0.5, 1.0])
def test_exp_action(dims, c, prec, tol):
    a, b, r, _ = make_case(dims)
    v0 = np.random.default_rng(4).standard_normal(tuple(dims[::-1]))
    tau = 2.5e-3
    prob = O.ADRProblem(dims, a, b, r)
    ctx = context(dims, tau, "lawson4", prec, a, b, r)
    dt = DTYPES[prec]
    fv, v = guarded(v0.shape, dt, v0)
    fy, y = guarded(v0.shape, dt)
    ctx.apply_exp(c, v, y)
    torch.cuda.synchronize()
    check_guards(fv)
    check_guards(fy)
    ref = O.MatrixFunctions(prob, tau).exp_action(c, v.double().cpu().numpy())
    assert_parity(y.cpu().numpy(), ref, tol, what=f"exp {dims} c={c} {prec}")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("dims", [(32, 32), (37, 29), (24, 24, 24), (31, 17, 22)])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_phi_action(dims, k, prec, tol):
    a, b, r, _ = make_case(dims)
    v0 = np.random.default_rng(6).standard_normal(tuple(dims[::-1]))
    tau = 2e-3
    prob = O.ADRProblem(dims, a, b, r)
    ctx = context(dims, tau, "etd2rk", prec, a, b, r)
    dt = DTYPES[prec]
    fv, v = guarded(v0.shape, dt, v0)
    fy, y = guarded(v0.shape, dt)
    ctx.apply_phi(k, v, y)
    torch.cuda.synchronize()
    check_guards(fy)
    vin = v.double().cpu().numpy()
    mf = O.MatrixFunctions(prob, tau)
    ref = mf.exp_action(1.0, vin) if k == 0 else mf.phi_action(k, 1.0, vin)
    assert_parity(y.cpu().numpy(), ref, tol, what=f"phi{k} {dims} {prec}")


INTEGRATE = [
    # (dims, b, scheme, T, m)
    ((32, 32), (10.0, 10.0), "lawson_euler", 0.1, 20),
    ((32, 32), (10.0, 10.0), "etd2rk", 0.1, 20),
    ((32, 32), (10.0, 10.0), "lawson4", 0.1, 20),
    ((41, 27), (6.0, -9.0), "etd2rk", 0.05, 10),
    ((20, 20, 20), (10.0, 10.0, 10.0), "etd2rk", 0.04, 8),
    ((24, 24, 24), (10.0, 10.0, 10.0), "lawson4", 0.04, 8),
    ((19, 26, 33), (3.0, -5.0, 8.0), "lawson_euler", 0.04, 8),
    ((19, 26, 33), (3.0, -5.0, 8.0), "lawson4", 0.04, 8),
] + [
    # the paper's other schemes (Appendix) on the same kernels
    case for scheme in ("exponential_euler", "erk2p1", "stabilized_lawson_euler", "lawson2a", "lawson2b",
                        "stabilized_lawson2")
    for case in (((37, 29), (6.0, -9.0), scheme, 0.05, 10), ((19, 26, 33), (3.0, -5.0, 8.0), scheme, 0.04, 8))
]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("dims,b,scheme,T,m", INTEGRATE)
def test_integrate_matches_oracle(dims, b, scheme, T, m, prec, tol):
    a, bb, r, u0 = make_case(dims, b=b)
    tau = T / m
    ctx = context(dims, tau, scheme, prec, a, bb, r)
    dt = DTYPES[prec]
    fu, u = guarded(u0.shape, dt, u0)
    ctx.integrate(u, 0.0, T, m)
    torch.cuda.synchronize()
    check_guards(fu)
    ref = O.solve(dims, a, bb, r, u0, tau, m, scheme)
    assert_parity(u.cpu().numpy(), ref, tol, what=f"{scheme} {dims} {prec}")


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("scheme", ["lawson_euler", "etd2rk", "lawson4"])
def test_graph_replay_equals_direct_steps_bitwise(scheme, prec):
    """adr_integrate (captured CUDA graphs on a non-default stream: an 8-step graph and a
    1-step graph for the rest) and m calls of adr_step give identical bits, for m below and
    above 8, and two runs are bitwise deterministic."""
    dims = (29, 23, 21) if prec == "fp64" else (64, 48, 40)
    a, b, r, u0 = make_case(dims)
    tau = 2e-3
    dt = torch.float64 if prec == "fp64" else torch.float32
    stream = torch.cuda.Stream()
    for m in (5, 19):
        with torch.cuda.stream(stream):
            ctx = adr.Context(dims, tau, scheme, prec, stream=stream)
            ctx.set_coeffs(a, b, r)
            u1 = torch.tensor(u0, dtype=dt, device="cuda")
            u2 = u1.clone()
            u3 = u1.clone()
            ctx.integrate(u1, 0.0, m * tau, m)
            for i in range(m):
                ctx.step(u2, i * tau)
            ctx.integrate(u3, 0.0, m * tau, m)
            ctx.synchronize()
        assert torch.equal(u1, u2) and torch.equal(u1, u3), m
        ctx.close()


def test_integrate_host_matches_device():
    dims = (32, 32)
    a, b, r, u0 = make_case(dims)
    ctx = context(dims, 5e-3, "etd2rk", "fp64", a, b, r)
    ud = torch.tensor(u0, device="cuda")
    uh = torch.tensor(u0).pin_memory()
    ctx.integrate(ud, 0.0, 0.1, 20)
    ctx.integrate_host(uh, 0.0, 0.1, 20)
    torch.cuda.synchronize()
    assert torch.equal(ud.cpu(), uh)


def test_config2_full_size_fp64():
    """3-D 128^3 FP64 ETD2RK, 50 steps to T = 0.1 (the full workload), against the oracle."""
    w = W.config2()
    ctx = context(w.dims, w.tau, w.scheme, "fp64", w.a_nodes, w.b, w.r_poly)
    u = torch.tensor(w.u0, device="cuda")
    ctx.integrate(u, 0.0, w.tau * w.m, w.m)
    torch.cuda.synchronize()
    ref = O.solve(w.dims, w.a_nodes, w.b, w.r_poly, w.u0, w.tau, w.m, w.scheme)
    err, err_inf, _ = assert_parity(u.cpu().numpy(), ref, 1e-12, what="128^3 etd2rk fp64")
    print(f"config2 128^3 etd2rk fp64 rel l2 {err:.3e}, rel max {err_inf:.3e}")


def test_state_errors():
    dims = (16, 16)
    ctx = adr.Context(dims, 1e-3, "etd2rk", "fp64", phi_route="eigen")
    u = torch.zeros(dims, dtype=torch.float64, device="cuda")
    with pytest.raises(adr.AdrError) as e:
        ctx.step(u)
    assert e.value.status == 7
    a, b, r, _ = make_case(dims)
    # cell Peclet number |b| h / (2 abar) >= 1: no real eigenbasis for the phi route
    with pytest.raises(adr.AdrError) as e:
        ctx.set_coeffs(a, (400.0, 0.0), r)
    assert e.value.status == 5
    # the same coefficients are fine for an exp-only (Lawson) scheme
    adr.Context(dims, 1e-3, "lawson4", "fp64").set_coeffs(a, (400.0, 0.0), r)
    # kappa guard
    ctx2 = adr.Context((64, 64), 1e-3, "etd2rk", "fp32", kappa_tol=1e-9, phi_route="eigen")
    with pytest.raises(adr.AdrError) as e:
        ctx2.set_coeffs(*make_case((64, 64))[:3])
    assert e.value.status == 4


# ----------------------------------------------------------------------------- phi doubling route
# Exponentials only: for eigenbases too ill-conditioned for the eigen route, or complex
# spectra (cell Peclet >= 1). The oracle's reference is its dense route (augmented-matrix
# exponential of the full Kronecker sum), valid for any conditioning on these small grids.
DOUBLING = [
    # (dims, b): prod kappa(V_mu) ~ 1e13 (2-D), complex spectrum (3-D, cell Peclet 1.2)
    ((24, 20), (52.0, -42.0)),
    ((10, 9, 8), (40.0, -30.0, 35.0)),
]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 5e-5)])
@pytest.mark.parametrize("dims,b", DOUBLING)
@pytest.mark.parametrize("k", [1, 2])
def test_phi_doubling_action_matches_dense_oracle(dims, b, k, prec, tol):
    a, bb, r, _ = make_case(dims, b=b)
    tau = 2e-3
    ctx = context(dims, tau, "etd2rk", prec, a, bb, r)
    route, halvings, terms = ctx.phi_route()
    assert route == "doubling" and halvings > 0 and terms > 0
    v0 = np.random.default_rng(12).standard_normal(tuple(dims[::-1]))
    dt = DTYPES[prec]
    fv, v = guarded(v0.shape, dt, v0)
    fy, y = guarded(v0.shape, dt)
    ctx.apply_phi(k, v, y)
    torch.cuda.synchronize()
    check_guards(fy)
    prob = O.ADRProblem(dims, a, bb, r)
    ref = O.MatrixFunctions(prob, tau).phi_action_dense(k, 1.0, v.double().cpu().numpy())
    assert_parity(y.cpu().numpy(), ref, tol, what=f"doubling phi{k} {dims} {prec}")


@pytest.mark.parametrize("scheme", ["etd2rk", "exponential_euler", "erk2p1"])
@pytest.mark.parametrize("dims,b", DOUBLING)
def test_phi_schemes_on_the_doubling_route_match_dense_oracle(dims, b, scheme):
    a, bb, r, u0 = make_case(dims, b=b)
    tau, m = 2e-3, 4
    ctx = context(dims, tau, scheme, "fp64", a, bb, r)
    fu, u = guarded(u0.shape, torch.float64, u0)
    ctx.integrate(u, 0.0, m * tau, m)
    torch.cuda.synchronize()
    check_guards(fu)
    ref = O.solve(dims, a, bb, r, u0, tau, m, scheme, phi_route="dense")
    # strongly non-normal operators (prod kappa ~ 1e13, or complex spectra): the oracle's
    # dense exponential of the augmented matrix and the doubling chain both carry errors of
    # order eps ||tau A|| times the non-normality, ~1e-12 after these steps
    assert_parity(u.cpu().numpy(), ref, 5e-12, what=f"doubling {scheme} {dims}")


def test_doubling_route_forced_on_a_well_conditioned_grid_matches_eigen_oracle():
    dims = (33, 30)
    a, bb, r, u0 = make_case(dims)
    tau, m = 3e-3, 6
    ctx = adr.Context(dims, tau, "etd2rk", "fp64", phi_route="doubling")
    ctx.set_coeffs(a, bb, r)
    assert ctx.phi_route()[0] == "doubling"
    u = torch.tensor(u0, dtype=torch.float64, device="cuda")
    ctx.integrate(u, 0.0, m * tau, m)
    ctx.synchronize()
    ref = O.solve(dims, a, bb, r, u0, tau, m, "etd2rk")
    assert_parity(u.cpu().numpy(), ref, 1e-12, what="forced doubling etd2rk")


# ----------------------------------------------------------------------------- lambda scan
def test_lambda_scan_errors_match_oracle():
    """Section 3's scan on a small grid: the library's error for each lambda equals the
    oracle's (the same scheme with that lambda against Lawson4 at tau/8), and the chosen
    lambda is the argmin."""
    dims = (24, 20)
    a, bb, r, u0 = make_case(dims, b=(10.0, -6.0))
    tau, m = 4e-3, 10
    lams = [0.25, 0.5, 0.75, 1.0]
    best, errs = adr.adr_lambda_scan(dims, tau, "lawson_euler", "fp64", a, bb, r, u0, m, lambdas=lams)
    ref = O.solve(dims, a, bb, r, u0, tau / 8, 8 * m, "lawson4")
    for lam, err in errs:
        got = O.solve(dims, a, bb, r, u0, tau, m, "lawson_euler", lam=lam)
        assert abs(err - O.rel_l2(got, ref)) <= 1e-6 * err, lam
    assert best == min(errs, key=lambda t: t[1])[0]
    # default candidates: from the Table 1 bound of the scheme to 1
    best2, errs2 = adr.adr_lambda_scan(dims, tau, "etd2rk", "fp64", a, bb, r, u0, m, n_lambdas=5)
    assert abs(errs2[0][0] - adr.adr_stability_bound("etd2rk")) < 1e-12 and errs2[-1][0] == 1.0
    assert all(np.isfinite(e) for _, e in errs2) and best2 == min(errs2, key=lambda t: t[1])[0]



# ------------------------------------------- the paper's 3-D problem form (Eq. (adr3d))
# a Lap u, Dirichlet faces at x_mu = 0, Neumann faces at x_mu = 1 (mirror ghosts, h = 1/n).
def mixed_case(dims, seed=21):
    rng = np.random.default_rng(seed)
    a = 0.05 + 0.1 * rng.random(tuple(n + 2 for n in dims[::-1]))
    b = (-1.0, 0.6, -0.3)[: len(dims)] + (0.0,) * (3 - len(dims))
    u0 = rng.standard_normal(tuple(dims[::-1])) * 0.1 + 0.3
    return a, b, (0.0, 1.0, 0.0, 1.0), u0


def mixed_context(dims, tau, scheme, prec, a, b, r, **kw):
    ctx = adr.Context(dims, tau, scheme, prec, bc="mixed", form="adelta", **kw)
    ctx.set_coeffs(a, b, r)
    return ctx


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
@pytest.mark.parametrize("dims", [(24, 20, 18), (25, 19, 17), (30, 26), (33, 21)])
def test_mixed_adelta_stencil_F_and_g(dims, prec, tol):
    a, b, r, u0 = mixed_case(dims)
    ctx = mixed_context(dims, 1e-3, "lawson4", prec, a, b, r)
    dt = DTYPES[prec]
    _, u = guarded(u0.shape, dt, u0)
    fF, F = guarded(u0.shape, dt)
    fg, g = guarded(u0.shape, dt)
    ctx.eval_rhs(u, F, g)
    torch.cuda.synchronize()
    check_guards(fF)
    check_guards(fg)
    prob = O.ADRProblem(dims, a, b, r, bc="mixed", form="adelta")
    uin = u.double().cpu().numpy()
    assert_parity(F.cpu().numpy(), prob.F(uin), tol, what=f"a Lap u F {dims} {prec}")
    assert_parity(g.cpu().numpy(), prob.g(uin), tol, what=f"a Lap u g {dims} {prec}")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
@pytest.mark.parametrize("dims", [(24, 20, 18), (132, 36, 20)])     # the second: TMA-staged FP32 kernel
def test_adelta_form_with_dirichlet_faces(prec, tol, dims):
    a, b, r, u0 = mixed_case(dims)
    ctx = adr.Context(dims, 1e-3, "lawson4", prec, form="adelta")
    ctx.set_coeffs(a, b, r)
    dt = DTYPES[prec]
    _, u = guarded(u0.shape, dt, u0)
    _, F = guarded(u0.shape, dt)
    ctx.eval_rhs(u, F, None)
    torch.cuda.synchronize()
    prob = O.ADRProblem(dims, a, b, r, form="adelta")
    assert_parity(F.cpu().numpy(), prob.F(u.double().cpu().numpy()), tol, what=f"a Lap u Dirichlet F {prec}")


@pytest.mark.parametrize("scheme", ["lawson4", "lawson2a", "lawson2b", "stabilized_lawson2", "lawson_euler"])
def test_mixed_adelta_lawson_schemes_match_oracle(scheme):
    dims = (24, 20, 18)
    a, b, r, u0 = mixed_case(dims)
    tau, m = 2e-3, 6
    ctx = mixed_context(dims, tau, scheme, "fp64", a, b, r)
    fu, u = guarded(u0.shape, torch.float64, u0)
    ctx.integrate(u, 0.0, m * tau, m)
    torch.cuda.synchronize()
    check_guards(fu)
    ref = O.solve(dims, a, b, r, u0, tau, m, scheme, bc="mixed", form="adelta")
    assert_parity(u.cpu().numpy(), ref, 1e-12, what=f"a Lap u {scheme}")


@pytest.mark.parametrize("scheme", ["etd2rk", "erk2p1"])
def test_mixed_adelta_phi_schemes_on_the_doubling_route(scheme):
    """No closed-form eigenbasis with Neumann rows: the phi schemes take the doubling route."""
    dims = (10, 9, 8)
    a, b, r, u0 = mixed_case(dims)
    tau, m = 2e-3, 4
    ctx = mixed_context(dims, tau, scheme, "fp64", a, b, r)
    assert ctx.phi_route()[0] == "doubling"
    fu, u = guarded(u0.shape, torch.float64, u0)
    ctx.integrate(u, 0.0, m * tau, m)
    torch.cuda.synchronize()
    check_guards(fu)
    ref = O.solve(dims, a, b, r, u0, tau, m, scheme, bc="mixed", form="adelta", phi_route="dense")
    assert_parity(u.cpu().numpy(), ref, 1e-12, what=f"a Lap u doubling {scheme}")


def test_e4_workload_fp64_and_mixed_precision_against_oracle():
    """The paper's three-dimensional experiment at N = 60 (b = -1), a few Lawson2a steps:
    FP64 to 1e-12, the tensor-core path to 1e-6."""
    w = W.config_e4(n=60, b=-1.0, scheme="lawson2a", m=32)
    steps = 4
    ref = O.solve(w.dims, w.a_nodes, w.b, w.r_poly, w.u0, w.tau, steps, w.scheme, bc="mixed", form="adelta")
    for prec, tol in (("fp64", 1e-12), ("bf16x3", 1e-6)):
        ctx = mixed_context(w.dims, w.tau, w.scheme, prec, w.a_nodes, w.b, w.r_poly)
        u = torch.tensor(w.u0, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
        ctx.integrate(u, 0.0, steps * w.tau, steps)
        ctx.synchronize()
        err, err_inf, _ = assert_parity(u.double().cpu().numpy(), ref, tol, what=f"E4 N=60 lawson2a {prec}")
        print(f"E4 N=60 lawson2a {prec}: {err:.3e}, max norm {err_inf:.3e}")


def test_neumann_faces_need_the_adelta_form():
    with pytest.raises(adr.AdrError) as e:
        adr.Context((16, 16), 1e-3, "lawson4", "fp64", bc="mixed", form="flux")
    assert e.value.status == 8


def test_e4_lambda_scan_on_the_gpu_chooses_the_papers_lambda():
    """Section 3's scan on the paper's 3-D experiment as Section 5.2 runs it (N = 2^4, m = 2^8,
    T = 1/4, b = -0.01, maximum norm), over the lambda values the paper printed for
    Lawson-Euler: the library chooses the printed argmin (0.356; the table of lambda values of
    Section 5.2 gives 0.36), and its errors are the printed ones within 1e-3 (its reference is
    Lawson4 at tau/16, the paper's Lawson2b at a small step)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "e4_lambda_scan_paper.json")))
    pts = g["points"]["-0.01"]["lawson_euler"]
    w = W.config_e4(n=16, b=-0.01, scheme="lawson_euler", m=256, T=0.25)
    best, errs = adr.adr_lambda_scan(w.dims, w.tau, "lawson_euler", "fp64", w.a_nodes, w.b, w.r_poly, w.u0, w.m,
                                     lambdas=[lam for lam, _ in pts], norm="max", ref_substeps=16,
                                     bc="mixed", form="adelta")
    assert best == min(pts, key=lambda t: t[1])[0]
    for (lam, err), (_, paper) in zip(errs, pts):
        assert abs(err / paper - 1.0) <= 1e-3, (lam, err, paper)

"""Periodic Fourier pseudospectral contexts (the paper's two-dimensional experiment form,
Section 5.1, Eq. (ad2d)) through the C ABI against the FP64 oracle's PeriodicProblem.

Tolerances (relative l2):
  * FP64 matrix-function actions 1e-12; F and g 1e-11: the spectral derivative multiplies
    the FFT's rounding (about 1e-16 log2 N relative to the coefficients) by up to k_max^2,
    k_max = (n/2)(2 pi / L), which is 1e2 to 1e3 on these grids.
  * FP64 time integration 1e-11 (the same amplification, once per step, damped by e^{tau A}).
  * FP32: 1e-4 on the full E3 horizon (256 steps at n = 256). Each FP32 transform leaves a
    rounding error of about eps32 log2(N) = 6e-8 x 16 = 1e-6 of the state spread over all modes;
    the flux divergence multiplies it by up to a^max k_max^2 (0.67 x 42.7^2 = 1.2e3) and the step
    by tau = 1/64, so each step adds about 2e-5 in the highest modes, which e^{tau A} then damps;
    random-walk accumulation over sqrt(256) = 16 steps' worth of surviving modes gives an
    estimate of 7e-5.
Grids include the largest line (n = 1024), the degenerate n = 2 direction (modes 0 and
Nyquist only), non-square 2-D and 3-D shapes.
"""
import numpy as np
import pytest

from oracle import adr_oracle as O
from parity import assert_parity
from paper_2303_15861_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2303_15861_gb300 import adr, build_lib  # noqa: E402

build_lib.build()
adr.load_library()

DT = {"fp64": torch.float64, "fp32": torch.float32}
SCHEMES = ["lawson_euler", "etd2rk", "lawson4", "exponential_euler", "erk2p1", "stabilized_lawson_euler",
           "lawson2a", "lawson2b", "stabilized_lawson2"]


def context(w, L, a_diag, b_field, prec="fp64", scheme=None, stream=None, lam=1.0):
    ctx = adr.Context(w.dims, w.tau, scheme or w.scheme, prec, stream=stream, periodic=True, length=L, lam=lam)
    ctx.set_coeffs_periodic(a_diag, b_field, w.r_poly)
    return ctx


def dev(x, prec="fp64"):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=DT[prec], device="cuda")


def host(t):
    return t.double().cpu().numpy()


@pytest.mark.parametrize("dims", [(32, 64), (1024, 4), (2, 64), (16, 8, 32), (4, 4, 4)])
def test_building_blocks_match_oracle(dims):
    """F, g, e^{c tau A} and phi_k(tau A) of a random state."""
    w, L, a, b = W.periodic_instance(dims, T=0.05, m=4)
    ctx = context(w, L, a, b, scheme="etd2rk")
    prob = O.PeriodicProblem(dims, L, a, b, w.r_poly)
    ops = O.PeriodicOps(prob, w.tau)
    v = np.random.default_rng(3).standard_normal(w.u0.shape)
    u = dev(w.u0)
    F = torch.empty_like(u)
    g = torch.empty_like(u)
    ctx.eval_rhs(u, F, g)
    y = {}
    for c in (0.5, 1.0):
        y[("exp", c)] = torch.empty_like(u)
        ctx.apply_exp(c, dev(v), y[("exp", c)])
    for k in (0, 1, 2):
        y[("phi", k)] = torch.empty_like(u)
        ctx.apply_phi(k, dev(v), y[("phi", k)])
    ctx.synchronize()
    assert_parity(host(F), ops.F(w.u0), 1e-11, what="periodic F")
    assert_parity(host(g), ops.g(w.u0), 1e-11, what="periodic g")
    for c in (0.5, 1.0):
        assert_parity(host(y[("exp", c)]), ops.expA(c, v), 1e-12, what=c)
    for k in (0, 1, 2):
        assert_parity(host(y[("phi", k)]), ops.phi(k, 1.0, v), 1e-12, what=k)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_fp64_schemes_match_oracle(scheme):
    w, L, a, b = W.periodic_instance((32, 16), scheme=scheme, T=0.2, m=6)
    ctx = context(w, L, a, b)
    u = dev(w.u0)
    ctx.integrate(u, 0.0, w.m * w.tau, w.m)
    ctx.synchronize()
    ref = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, w.tau, w.m, scheme)
    assert_parity(host(u), ref, 1e-11)


@pytest.mark.parametrize("scheme", ["lawson4", "etd2rk", "stabilized_lawson2"])
def test_fp64_3d_matches_oracle(scheme):
    w, L, a, b = W.periodic_instance((16, 32, 8), scheme=scheme, T=0.1, m=4)
    ctx = context(w, L, a, b, lam=0.8)
    u = dev(w.u0)
    ctx.integrate(u, 0.0, w.m * w.tau, w.m)
    ctx.synchronize()
    ref = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, w.tau, w.m, scheme, lam=0.8)
    assert_parity(host(u), ref, 1e-11)


def test_e3_workload_fp64_matches_oracle():
    """The paper's 2-D experiment at n = 128, 64 steps to T = 1 (Lawson2a)."""
    w, L, a, b = W.config_e3(n=128, scheme="lawson2a", m=64, T=1.0)
    ctx = context(w, L, a, b)
    u = dev(w.u0)
    ctx.integrate(u, 0.0, w.m * w.tau, w.m)
    ctx.synchronize()
    ref = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, w.tau, w.m, "lawson2a")
    assert_parity(host(u), ref, 1e-11)


@pytest.mark.parametrize("scheme", ["lawson2a", "etd2rk"])
def test_e3_workload_fp32_full_horizon(scheme):
    """The full E3 workload (n = 256, 256 steps to T = 4) in FP32 against the FP64 oracle."""
    w, L, a, b = W.config_e3(n=256, scheme=scheme)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = context(w, L, a, b, prec="fp32", stream=s)
        u = dev(w.u0, "fp32")
        ctx.integrate(u, 0.0, w.m * w.tau, w.m)
        ctx.synchronize()
    ref = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, w.tau, w.m, scheme)
    err, err_inf, _ = assert_parity(host(u), ref, 1e-4, what=f"E3 n=256 {scheme} fp32")
    print(f"E3 n=256 {scheme} fp32: rel l2 {err:.3e}, max norm {err_inf:.3e}")


def test_graph_replay_equals_direct_steps():
    w, L, a, b = W.periodic_instance((64, 32), scheme="lawson4", m=3)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = context(w, L, a, b, prec="fp32", stream=s)
        u1 = dev(w.u0, "fp32")
        u2 = u1.clone()
        ctx.integrate(u1, 0.0, 3 * w.tau, 3)
        for i in range(3):
            ctx.step(u2, i * w.tau)
        ctx.synchronize()
    assert torch.equal(u1, u2)


def test_integrate_host_equals_device():
    w, L, a, b = W.periodic_instance((64, 32), scheme="etd2rk", m=2)
    ctx = context(w, L, a, b)
    u = dev(w.u0)
    h = u.cpu().pin_memory()
    ctx.integrate(u, 0.0, 2 * w.tau, 2)
    ctx.integrate_host(h, 0.0, 2 * w.tau, 2)
    ctx.synchronize()
    assert torch.equal(u.cpu(), h)


def test_context_facts_and_launch_count():
    w, L, a, b = W.periodic_instance((32, 16), scheme="etd2rk")
    ctx = context(w, L, a, b)
    assert ctx.phi_route()[0] == "fourier"
    info = ctx.info()
    assert info["kappa"][:2] == [1.0, 1.0]
    assert info["abar"] == pytest.approx(max(x.max() for x in a))
    assert info["beta"][0] == pytest.approx(b[0].mean()) and info["beta"][1] == pytest.approx(b[1].mean())
    # 2-D: every stage is kept in Fourier space from the state's transform to the stage result,
    # five passes (instead of a right-hand side of 5 passes and multipliers of 3), four for a
    # stage that starts from the previous stage's result; Lawson4 and stabilized Lawson2 keep the
    # right-hand side and multiplier passes
    assert ctx.kernels_per_step() == 5 + 4
    ops = ctx.profile_step(dev(w.u0))
    assert [k for k, _ in ops] == [8, 8]
    w3, L3, a3, b3 = W.periodic_instance((8, 16, 8), scheme="lawson2a")
    ctx3 = context(w3, L3, a3, b3)
    assert ctx3.kernels_per_step() == 2 * 9 + 3 * 5   # 3-D: 9 and 5 passes
    fused = {"lawson2a": 2, "lawson_euler": 1, "etd2rk": 2, "erk2p1": 2, "exponential_euler": 1,
             "stabilized_lawson_euler": 1, "lawson2b": 2}
    for scheme, stages in fused.items():
        w2, L2, a2, b2 = W.periodic_instance((32, 16), scheme=scheme)
        assert context(w2, L2, a2, b2).kernels_per_step() == 5 * stages - (stages - 1), scheme
    w4, L4, a4, b4 = W.periodic_instance((32, 16), scheme="lawson4")
    c4 = context(w4, L4, a4, b4)
    assert 8 not in [k for k, _ in c4.profile_step(dev(w4.u0))]


def test_periodic_context_refuses_grid_coefficients_and_unset_steps():
    w, L, a, b = W.periodic_instance((16, 16), scheme="lawson2a")
    ctx = adr.Context(w.dims, w.tau, "lawson2a", "fp64", periodic=True, length=L)
    u = dev(w.u0)
    with pytest.raises(adr.AdrError) as e:
        ctx.step(u)
    assert e.value.status == 7
    with pytest.raises(adr.AdrError) as e:
        ctx.set_coeffs(np.ones((18, 18)), (0.0, 0.0), w.r_poly)
    assert e.value.status == 1
    with pytest.raises(adr.AdrError) as e:   # non-finite coefficient
        bad = [a[0].copy(), a[1]]
        bad[0][3, 4] = np.nan
        ctx.set_coeffs_periodic(bad, b, w.r_poly)
    assert e.value.status == 1
    ctx.set_coeffs_periodic(a, b, w.r_poly)
    ctx.step(u)
    ctx.synchronize()


def test_periodic_lambda_scan_reproduces_the_papers_choice():
    """Section 3's scan on the paper's 2-D experiment as Section 5.1 runs it (2^6 modes, 2^8
    steps to T = 4, relative maximum-norm errors), over the lambda values the paper printed for
    Lawson-Euler: the library's errors equal the oracle's (the same scheme against Lawson4 at
    tau/8), and the chosen lambda is the paper's (0.218; the table of lambda values gives 0.22)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "e3_lambda_scan_paper.json")))
    lams = [lam for lam, _ in g["points"]["lawson_euler"]]
    w, L, a, b = W.config_e3(n=64, scheme="lawson_euler", m=256, T=4.0)
    best, errs = adr.adr_lambda_scan_periodic(w.dims, L, w.tau, "lawson_euler", "fp64", a, b, w.r_poly, w.u0, w.m,
                                              lambdas=lams, norm="max")
    assert best == 0.218
    ref = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, w.tau / 8, 8 * w.m, "lawson4")
    for lam, err in (errs[0], errs[7], errs[-1]):
        got = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, w.tau, w.m, "lawson_euler", lam=lam)
        want = np.abs(got - ref).max() / np.abs(ref).max()
        assert abs(err - want) <= 1e-6 * want, (lam, err, want)


def test_e2_on_an_embedded_grid_matches_the_1d_oracle_and_the_paper():
    """The paper's one-dimensional problem (Section 4, Eq. (adnonlinear)) on n x 2 Fourier nodes,
    constant along x2: Lawson-Euler at lambda = 0.218 with the paper's 2^12 steps to T = 1/10 in
    FP64. The two rows stay equal, the x1 line equals the 1-D oracle, and its error against a
    converged reference is the paper's printed 2.574e-4 (the figure of errors against lambda)
    within 1%."""
    w, L, a, b = W.config_e2(embed=True, scheme="lawson_euler")
    ctx = context(w, L, a, b, lam=0.218)
    u = dev(w.u0)
    ctx.integrate(u, 0.0, w.m * w.tau, w.m)
    ctx.synchronize()
    h = host(u)
    assert np.allclose(h[0], h[1], rtol=0, atol=1e-15)
    w1, L1, a1, b1 = W.config_e2(scheme="lawson_euler")
    ref1 = O.solve_periodic(w1.dims, L1, a1, b1, w1.r_poly, w1.u0, w1.tau, w1.m, "lawson_euler", lam=0.218)
    assert_parity(h[0], ref1, 1e-11)
    conv = O.solve_periodic(w1.dims, L1, a1, b1, w1.r_poly, w1.u0, w1.tau / 4, 4 * w1.m, "lawson4")
    err = np.abs(h[0] - conv).max() / np.abs(conv).max()
    assert abs(err / 2.57438011667187e-04 - 1.0) < 0.01, err


@pytest.mark.parametrize("dims", [(32, 64), (64, 2), (16, 8, 32)])
def test_adelta_building_blocks_match_oracle(dims):
    """The a Lap u form (Section 4, Eq. (adlinearzero), with advection and reaction added):
    F and g against the oracle."""
    w, L, a, b = W.periodic_instance(dims, T=0.05, m=4)
    ctx = adr.Context(w.dims, w.tau, "etd2rk", "fp64", periodic=True, length=L, form="adelta")
    ctx.set_coeffs_periodic(a, b, w.r_poly)
    prob = O.PeriodicProblem(dims, L, a, b, w.r_poly, form="adelta")
    u = dev(w.u0)
    F = torch.empty_like(u)
    g = torch.empty_like(u)
    ctx.eval_rhs(u, F, g)
    ctx.synchronize()
    assert_parity(host(F), prob.F(w.u0), 1e-11)
    assert_parity(host(g), prob.g(w.u0), 1e-11)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_fp64_schemes_in_the_adelta_form_match_oracle(scheme):
    """Every scheme in the a Lap u form (the Fourier-space stages then carry the a Lap u product
    with r(u) in the transformed pointwise part), on a non-square grid, lambda = 0.8."""
    w, L, a, b = W.periodic_instance((16, 32), scheme=scheme, T=0.1, m=5)
    ctx = adr.Context(w.dims, w.tau, scheme, "fp64", periodic=True, length=L, form="adelta", lam=0.8)
    ctx.set_coeffs_periodic(a, b, w.r_poly)
    u = dev(w.u0)
    ctx.integrate(u, 0.0, w.m * w.tau, w.m)
    ctx.synchronize()
    ref = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, w.tau, w.m, scheme, lam=0.8, form="adelta")
    assert_parity(host(u), ref, 1e-11, what=scheme)


@pytest.mark.parametrize("scheme", ["erk2p1", "lawson2b", "exponential_euler", "stabilized_lawson_euler"])
def test_fp32_fused_schemes_match_oracle(scheme):
    """FP32 Fourier-space stages at n = 128 over 32 steps against the FP64 oracle (the FP32
    bound of the module docstring, on a shorter horizon)."""
    w, L, a, b = W.config_e3(n=128, scheme=scheme, m=32, T=0.5)
    ctx = context(w, L, a, b, prec="fp32")
    u = dev(w.u0, "fp32")
    ctx.integrate(u, 0.0, w.m * w.tau, w.m)
    ctx.synchronize()
    ref = O.solve_periodic(w.dims, L, a, b, w.r_poly, w.u0, w.tau, w.m, scheme)
    assert_parity(host(u), ref, 1e-4, what=f"fp32 {scheme}")


@pytest.mark.parametrize("scheme,lam,m,paper", [("lawson_euler", 1.0, 64, 0.00288149591423319),
                                                ("stabilized_lawson_euler", 1.0, 16, 0.00423707305496343),
                                                ("exponential_euler", 1.0, 16, 0.00192512919614741)])
def test_e1_on_an_embedded_grid_matches_the_paper(scheme, lam, m, paper):
    """The paper's linear experiment (Section 4, Eq. (adlinearzero)) at its 2^12 modes on
    4096 x 2 nodes in FP64: the error against the exact semidiscrete solution is the printed one
    (the figure of errors against m, panel lambda = 1) within 0.1%, and the x1 line equals the
    1-D oracle."""
    w, L, a, b = W.config_e1(scheme=scheme, m=m, embed=True)
    ctx = adr.Context(w.dims, w.tau, scheme, "fp64", periodic=True, length=L, form="adelta", lam=lam)
    ctx.set_coeffs_periodic(a, b, w.r_poly)
    u = dev(w.u0)
    ctx.integrate(u, 0.0, w.m * w.tau, w.m)
    ctx.synchronize()
    h = host(u)
    w1, L1, a1, b1 = W.config_e1(scheme=scheme, m=m)
    ref1 = O.solve_periodic(w1.dims, L1, a1, b1, w1.r_poly, w1.u0, w1.tau, w1.m, scheme, lam=lam, form="adelta")
    assert_parity(h[0], ref1, 1e-11)
    exact = O.periodic_linear_exact(O.PeriodicProblem(w1.dims, L1, a1, b1, w1.r_poly, form="adelta"), w1.u0,
                                    w1.m * w1.tau)
    err = np.abs(h[0] - exact).max() / np.abs(exact).max()
    assert abs(err / paper - 1.0) < 1e-3, err


@pytest.mark.parametrize("scheme,paper", [("lawson_euler", 0.00719585866877569), ("lawson2a", 4.76308840101909e-05)])
def test_e3_at_2_to_the_8_modes_reproduces_the_papers_error(scheme, paper):
    """The paper's 2-D experiment at N = 2^8, 2^8 steps to T = 4, lambda = 1 (Section 5.1, the
    bottom panels of the figure of errors against lambda), entirely on the GPU in FP64: the error
    in the maximum norm relative to a Lawson4 reference with 2^11 steps is the printed one within
    0.3%."""
    w, L, a, b = W.config_e3(n=256, scheme=scheme)
    ctx = context(w, L, a, b)
    u = dev(w.u0)
    ctx.integrate(u, 0.0, w.m * w.tau, w.m)
    wr, _, _, _ = W.config_e3(n=256, scheme="lawson4", m=2048)
    rc = context(wr, L, a, b)
    ur = dev(wr.u0)
    rc.integrate(ur, 0.0, wr.m * wr.tau, wr.m)
    ctx.synchronize()
    rc.synchronize()
    got, ref = host(u), host(ur)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert abs(err / paper - 1.0) < 3e-3, err

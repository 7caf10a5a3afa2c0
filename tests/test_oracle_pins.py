"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form, an
independent library routine on a different algorithm, high-precision arithmetic,
brute force on tiny grids, values printed in the paper, or observed convergence orders.
"""
import json
import os

import mpmath
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import adr_oracle as O
from paper_2303_15861_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- phi
@pytest.mark.parametrize("k", [1, 2])
def test_phi_matches_high_precision(k):
    """phi_1 = (e^z-1)/z and phi_2 = (phi_1-1)/z (Section 1, Theorem 2.4) in 50 digits."""
    mpmath.mp.dps = 50
    zs = np.concatenate([-np.logspace(-12, 5, 200), np.logspace(-12, 1, 60), [0.0, -1.0, 1.0]])
    got = O.phi(k, zs)
    for z, g in zip(zs, got):
        zz = mpmath.mpf(float(z))
        if zz == 0:
            ref = mpmath.mpf(1) / mpmath.factorial(k)
        elif k == 1:
            ref = mpmath.expm1(zz) / zz
        else:
            ref = (mpmath.expm1(zz) - zz) / (zz * zz)
        assert abs(g - float(ref)) <= 1e-15 * abs(float(ref)), (k, z, g, float(ref))


# ----------------------------------------------------------------------------- expm
def _toeplitz_tridiag(n, sub, diag, sup):
    return np.diag(np.full(n, diag)) + np.diag(np.full(n - 1, sup), 1) + np.diag(np.full(n - 1, sub), -1)


@pytest.mark.parametrize("scale", [1e-3, 0.3, 5.0, 80.0, 3000.0])
def test_expm_matches_scipy(scale):
    """Own [13/13] Pade scaling-and-squaring against scipy's implementation."""
    rng = np.random.default_rng(1)
    A = rng.standard_normal((24, 24)) * scale / 24
    ref = sla.expm(A)
    assert np.abs(O.expm(A) - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())


def test_expm_matches_mpmath_taylor():
    """Against mpmath's multiprecision matrix exponential on a small nonnormal matrix."""
    mpmath.mp.dps = 40
    A = np.array([[-3.0, 2.5, 0.0], [0.2, -4.0, 1.7], [0.0, 0.9, -2.0]])
    ref = np.array(mpmath.expm(mpmath.matrix(A.tolist())).tolist(), dtype=float)
    assert np.abs(O.expm(A) - ref).max() <= 2e-15


def test_expm_factor_matches_closed_form_eigen():
    """e^{tau A_mu} of the tridiagonal Toeplitz factor equals V e^{tau Lambda} V^-1 with the
    textbook eigenpairs lambda_j = d + 2 sqrt(sp) cos(j pi/(n+1)),
    v_j(i) = (s/p)^{i/2} sin(i j pi/(n+1))."""
    n, abar, beta = 30, 1.3, 7.0
    h = 1.0 / (n + 1)
    s, d, p = abar / h**2 - beta / (2 * h), -2 * abar / h**2, abar / h**2 + beta / (2 * h)
    A = _toeplitz_tridiag(n, s, d, p)
    j = np.arange(1, n + 1)
    lam = d + 2 * np.sqrt(s * p) * np.cos(j * np.pi / (n + 1))
    i = np.arange(1, n + 1)[:, None]
    V = (s / p) ** (i / 2.0) * np.sin(i * j[None, :] * np.pi / (n + 1))
    Vinv = (2.0 / (n + 1)) * np.sin(j[:, None] * i.T * np.pi / (n + 1)) * (s / p) ** (-i.T / 2.0)
    assert np.abs(V @ Vinv - np.eye(n)).max() < 1e-12
    tau = 2e-3
    ref = (V * np.exp(tau * lam)) @ Vinv
    assert np.abs(O.expm(tau * A) - ref).max() < 1e-13


def test_numpy_eig_matches_closed_form():
    """The oracle's eigen route (numpy.linalg.eig) against the closed-form spectrum."""
    w = W.config1()
    prob = O.ADRProblem(w.dims, w.a_nodes, w.b, w.r_poly)
    mf = O.MatrixFunctions(prob, w.tau)
    n = w.dims[0]
    h = 1.0 / (n + 1)
    for mu, (lam, V, Vi) in enumerate(mf.eig(), start=1):
        s = prob.abar / h**2 - prob.beta[mu - 1] / (2 * h)
        p = prob.abar / h**2 + prob.beta[mu - 1] / (2 * h)
        j = np.arange(1, n + 1)
        ref = np.sort(-2 * prob.abar / h**2 + 2 * np.sqrt(s * p) * np.cos(j * np.pi / (n + 1)))
        assert np.allclose(np.sort(lam), ref, rtol=1e-12, atol=1e-9)
        assert np.abs(V @ Vi - np.eye(n)).max() < 1e-11


# ----------------------------------------------------------------------------- Kronecker sum
def test_kron_sum_exp_identity():
    """exp(A_2 (+) A_1) = exp(A_2) (x) exp(A_1), with A_2 (+) A_1 := A_2 (x) I + I (x) A_1."""
    rng = np.random.default_rng(3)
    A1 = rng.standard_normal((5, 5))
    A2 = rng.standard_normal((4, 4))
    S = np.kron(A2, np.eye(5)) + np.kron(np.eye(4), A1)
    assert np.allclose(O.kron_sum_dense([A1, A2]), S, atol=0, rtol=0)
    assert np.abs(sla.expm(S) - np.kron(sla.expm(A2), sla.expm(A1))).max() < 1e-12


@pytest.mark.parametrize("dims", [(7, 5), (4, 5, 3)])
def test_mumode_exp_matches_dense_expm(dims):
    """mu-mode action of e^{c tau A} against scipy's expm of the full Kronecker sum."""
    a = W.sine_product_coefficient(dims)
    prob = O.ADRProblem(dims, a, (3.0, -2.0, 1.0), W.REACTION_U2_1MU)
    tau = 3e-3
    mf = O.MatrixFunctions(prob, tau)
    A = O.kron_sum_dense([prob.factor(mu) for mu in range(1, len(dims) + 1)])
    v = np.random.default_rng(0).standard_normal(tuple(dims[::-1]))
    for c in (0.5, 1.0):
        ref = sla.expm(c * tau * A) @ v.ravel()
        got = mf.exp_action(c, v).ravel()
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("dims", [(6, 5), (3, 4, 5)])
@pytest.mark.parametrize("k", [1, 2])
def test_phi_action_matches_augmented_expm(dims, k):
    """phi_k(tau A) v from the eigen route against the top-right block of the exponential
    of the augmented matrix [[tau A, v, 0], [0, 0, 1], [0, 0, 0]] (Al-Mohy & Higham)."""
    a = W.sine_product_coefficient(dims)
    prob = O.ADRProblem(dims, a, (4.0, 2.0, -3.0), W.REACTION_U2_1MU)
    tau = 4e-3
    A = O.kron_sum_dense([prob.factor(mu) for mu in range(1, len(dims) + 1)])
    v = np.random.default_rng(5).standard_normal(tuple(dims[::-1]))
    N = v.size
    Z = np.zeros((N + 2, N + 2))
    Z[:N, :N] = tau * A
    Z[:N, N] = v.ravel()
    Z[N, N + 1] = 1.0
    big = sla.expm(Z)
    ref = big[:N, N + k - 1]
    got = O.MatrixFunctions(prob, tau).phi_action(k, 1.0, v).ravel()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_dense_phi_route_matches_eigen_route_and_closed_forms(k):
    """The dense route (augmented-matrix exponential of the full Kronecker sum) agrees with
    the eigen route where that one is well conditioned, and with the scalar closed forms
    of phi_k on a 1-point-per-direction grid (A is then the scalar sum of the diagonals)."""
    dims = (5, 4, 3)
    a = W.sine_product_coefficient(dims)
    prob = O.ADRProblem(dims, a, (4.0, 2.0, -3.0), W.REACTION_U2_1MU)
    tau = 4e-3
    v = np.random.default_rng(9).standard_normal(tuple(dims[::-1]))
    mf = O.MatrixFunctions(prob, tau)
    eig = mf.exp_action(1.0, v) if k == 0 else mf.phi_action(k, 1.0, v)
    dense = mf.phi_action_dense(k, 1.0, v)
    assert np.linalg.norm(dense - eig) <= 1e-12 * np.linalg.norm(eig)
    # scalar: one interior node per direction, A = sum of the three diagonal entries
    one = O.ADRProblem((1, 1, 1), np.ones((3, 3, 3)), (0.0, 0.0, 0.0), W.REACTION_U2_1MU)
    z = tau * sum(one.factor(mu)[0, 0] for mu in (1, 2, 3))
    closed = {0: np.exp(z), 1: np.expm1(z) / z, 2: (np.expm1(z) - z) / z**2}[k]
    got = O.MatrixFunctions(one, tau).phi_action_dense(k, 1.0, np.ones((1, 1, 1)))
    assert abs(got.item() - closed) <= 1e-12 * abs(closed)


def test_dense_phi_route_handles_an_ill_conditioned_eigenbasis():
    """With strong advection (cell Peclet 0.8) the eigenvector matrices have condition
    number ~1e13 per direction and the eigen route loses every digit; the dense route
    still meets the defining identity A phi_1(A) v = (e^A - I) v."""
    dims = (24, 20)
    a = np.ones((22, 26))
    prob = O.ADRProblem(dims, a, (52.0, -42.0), W.REACTION_U2_1MU)
    tau = 2e-3
    v = np.random.default_rng(3).standard_normal((20, 24))
    mf = O.MatrixFunctions(prob, tau)
    p1 = mf.phi_action_dense(1, 1.0, v)
    A = O.kron_sum_dense([prob.factor(1), prob.factor(2)])
    lhs = tau * (A @ p1.ravel())
    rhs = mf.phi_action_dense(0, 1.0, v).ravel() - v.ravel()
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)
    p2 = mf.phi_action_dense(2, 1.0, v)
    # phi_1(z) = 1 + z phi_2(z)
    assert np.linalg.norm(p1.ravel() - v.ravel() - tau * (A @ p2.ravel())) <= 1e-12 * np.linalg.norm(p1)


# ----------------------------------------------------------------------------- stencils
def _polynomial_case(d):
    dims = (9, 8, 7)[:d]
    nodes = W.mesh(dims, True)
    a = 1.0 + 0.3 * nodes[0] + 0.2 * nodes[1] + 0.05 * nodes[0] * nodes[1]
    if d == 3:
        a = a + 0.1 * nodes[2] + 0.07 * nodes[1] * nodes[2]
    return dims, a


@pytest.mark.parametrize("d", [2, 3])
def test_stencil_exact_on_polynomials(d):
    """Second-order centred flux form is exact when a is affine in each direction and
    u = prod x_mu (1 - x_mu): F_h(u) equals div(a grad u) + b.grad u + r(u) at the nodes."""
    dims, a_nodes = _polynomial_case(d)
    b = (2.0, -1.5, 0.7)[:d]
    r = (0.1, -0.4, 1.0, -1.0)
    prob = O.ADRProblem(dims, a_nodes, b, r)
    x = W.mesh(dims, False)
    q = [xi * (1 - xi) for xi in x]
    u = np.prod(q, axis=0)
    # analytic pieces
    if d == 2:
        ax = [0.3 + 0.05 * x[1], 0.2 + 0.05 * x[0]]
        aval = 1.0 + 0.3 * x[0] + 0.2 * x[1] + 0.05 * x[0] * x[1]
    else:
        ax = [0.3 + 0.05 * x[1], 0.2 + 0.05 * x[0] + 0.07 * x[2], 0.1 + 0.07 * x[1]]
        aval = 1.0 + 0.3 * x[0] + 0.2 * x[1] + 0.05 * x[0] * x[1] + 0.1 * x[2] + 0.07 * x[1] * x[2]
    F = np.zeros_like(u)
    for mu in range(d):
        others = np.prod([q[nu] for nu in range(d) if nu != mu], axis=0)
        du = (1 - 2 * x[mu]) * others
        ddu = -2.0 * others
        F += ax[mu] * du + aval * ddu + b[mu] * du
    F += r[0] + r[1] * u + r[2] * u**2 + r[3] * u**3
    assert np.abs(prob.F(u) - F).max() <= 1e-10 * np.abs(F).max()


@pytest.mark.parametrize("dims", [(8, 6), (5, 6, 4)])
def test_splitting_F_minus_Au_equals_g(dims):
    """g of Eq. (nonlin), computed directly, equals F(u) - A u with A the dense Kronecker
    sum of the 1-D factors of Eq. (linop) (brute force)."""
    a = W.sine_product_coefficient(dims, c=0.7, k=2) + 0.3 * W.mesh(dims, True)[0]
    prob = O.ADRProblem(dims, a, (5.0, -3.0, 2.0), (0.2, 0.5, 1.0, -1.0))
    u = np.random.default_rng(2).standard_normal(tuple(dims[::-1]))
    A = O.kron_sum_dense([prob.factor(mu) for mu in range(1, len(dims) + 1)])
    lhs = prob.F(u).ravel() - A @ u.ravel()
    assert np.abs(lhs - prob.g(u).ravel()).max() <= 1e-12 * np.abs(lhs).max()


def test_amax_beta_reading():
    """Eq. (amaxbeta): a_max = max of the nodal a; beta_mu = b_mu + mean of d_mu a.
    For a affine in x1 with slope 0.3 the mean of d_1 a is exactly 0.3; for the
    periodic sine product it is 0, so beta = b."""
    dims = (6, 5)
    x = W.mesh(dims, True)
    a = 1.0 + 0.3 * x[0] + 0.1 * np.sin(np.pi * x[1])
    prob = O.ADRProblem(dims, a, (1.0, 2.0), W.REACTION_U2_1MU)
    assert abs(prob.beta[0] - 1.3) < 1e-14 and abs(prob.beta[1] - 2.0) < 1e-14
    assert prob.abar == a.max()
    w = W.config1()
    prob = O.ADRProblem(w.dims, w.a_nodes, w.b, w.r_poly)
    assert np.allclose(prob.beta, [10.0, 10.0], rtol=0, atol=1e-13)
    # config-1 nodal maximum is below the analytic 1.5 (32 nodes do not hit the peak)
    assert 1.49 < prob.abar < 1.5


# ----------------------------------------------------------------------------- integrators
EXACT_FOR_LINEAR = ["lawson_euler", "etd2rk", "lawson4", "exponential_euler", "erk2p1",
                    "lawson2a", "lawson2b"]


@pytest.mark.parametrize("scheme", EXACT_FOR_LINEAR)
@pytest.mark.parametrize("dims", [(12, 10), (6, 5, 7)])
def test_exact_decay_of_discrete_eigenmodes(scheme, dims):
    """With g = 0 (a constant = a_max, r = 0) every scheme except the stabilized Lawson ones
    is exact for the linear problem (remark after Table 1): a discrete sine eigenmode
    decays as exp(t * sum_mu lambda_mu) exactly."""
    d = len(dims)
    abar = 1.7
    a = np.full(tuple(n + 2 for n in dims[::-1]), abar)
    b = (6.0, -4.0, 3.0)[:d]
    prob = O.ADRProblem(dims, a, b, (0.0, 0.0, 0.0, 0.0))
    modes, lam_total = [], 0.0
    for mu, (n, j) in enumerate(zip(dims, (1, 2, 3)), start=1):
        h = 1.0 / (n + 1)
        s = abar / h**2 - b[mu - 1] / (2 * h)
        p = abar / h**2 + b[mu - 1] / (2 * h)
        i = np.arange(1, n + 1)
        modes.append((s / p) ** (i / 2.0) * np.sin(i * j * np.pi / (n + 1)))
        lam_total += -2 * abar / h**2 + 2 * np.sqrt(s * p) * np.cos(j * np.pi / (n + 1))
    u0 = modes[0]
    for v in modes[1:]:
        u0 = np.multiply.outer(v, u0)
    T, m = 0.01, 7
    got = O.integrate(O.GridOps(prob, T / m), u0, m, scheme)
    ref = np.exp(lam_total * T) * u0
    assert O.rel_l2(got, ref) < 1e-12


@pytest.mark.parametrize("scheme", ["stabilized_lawson_euler", "stabilized_lawson2"])
def test_stabilized_lawson_not_exact_for_linear(scheme):
    """The same remark: the stabilized Lawson schemes are not exact for linear problems."""
    ops = O.ScalarOps(-3.0, lambda u: 0.0 * u, 0.1)
    got = O.SCHEMES[scheme](ops, np.array(1.0))
    assert abs(got - np.exp(-0.3)) > 1e-4


def _stability_function(scheme, z, lam):
    ops = O.ScalarOps(lam * z, lambda u: (1.0 - lam) * z * u, 1.0)
    return O.SCHEMES[scheme](ops, np.ones_like(z))


def test_stability_functions_match_paper():
    """One step of each oracle scheme on u' = lam z u + (1-lam) z u reproduces the stability
    functions printed in Theorems 2.1-2.7."""
    z = -np.concatenate([np.logspace(-3, 3, 41), [0.0]])
    p1, p2 = (lambda x: O.phi(1, x)), (lambda x: O.phi(2, x))
    for lam in (0.2, 0.35, 0.6, 1.0):
        e = np.exp(lam * z)
        printed = {
            "exponential_euler": 1 - 1 / lam + np.exp(z * lam) / lam,                    # Thm 2.1
            "lawson_euler": e * (1 + (1 - lam) * z),                                      # Thm 2.2
            "stabilized_lawson_euler": 1 + z * e,                                         # Thm 2.3
            "etd2rk": 1 + z * p1(lam * z) + z**2 * (1 - lam) * p2(lam * z) * p1(lam * z),  # Thm 2.4, c2=1
            "erk2p1": 1 + z * p1(lam * z) + z**2 / 2 * (1 - lam) * p1(lam * z) ** 2,      # Thm 2.5, c2=1
            "lawson2a": e * (1 + z * (1 - lam) * (1 + z * (1 - lam) / 2)),               # Thm 2.6
            "lawson2b": e * (1 + z / 2 * (1 - lam) + z / 2 * (1 - lam) * (1 + z * (1 - lam))),
            "stabilized_lawson2": 1 + z * np.exp(lam * z / 2)
            + z**2 / 2 * (1 - lam) * np.exp((1 + 0.327) * lam * z),                       # Thm 2.7
        }
        for scheme, ref in printed.items():
            got = _stability_function(scheme, z, lam)
            assert np.allclose(got, ref, rtol=1e-12, atol=1e-12), (scheme, lam)


def _lower_bound(scheme):
    z = -np.concatenate([np.logspace(-6, 7, 100001), np.linspace(0.0, 50.0, 100001)])
    lo, hi = 0.0, 1.0
    for _ in range(30):
        mid = 0.5 * (lo + hi)
        if np.all(np.abs(_stability_function(scheme, z, mid)) <= 1 + 1e-12):
            hi = mid
        else:
            lo = mid
    return hi


def test_table1_stability_bounds():
    """Bisection for the smallest unconditionally stable lambda reproduces Table 1."""
    with open(os.path.join(GOLDEN, "table1_stability_bounds.json")) as f:
        gold = json.load(f)
    for scheme, ref in gold["bounds"].items():
        assert abs(_lower_bound(scheme) - ref) <= gold["tolerance"], scheme


ORDERS = {"lawson_euler": 1, "exponential_euler": 1, "stabilized_lawson_euler": 1,
          "etd2rk": 2, "erk2p1": 2, "lawson2a": 2, "lawson2b": 2, "stabilized_lawson2": 2,
          "lawson4": 4}


def test_scalar_convergence_orders():
    """Non-stiff scalar Bernoulli equation u' = L u + u^2 with the exact solution
    u(t) = L u0 e^{Lt} / (L + u0 (1 - e^{Lt})): each scheme shows its classical order."""
    L, u0, T = -2.0, 0.7, 1.0
    exact = L * u0 * np.exp(L * T) / (L + u0 * (1 - np.exp(L * T)))
    for scheme, order in ORDERS.items():
        errs = []
        ms = (16, 32, 64)
        for m in ms:
            ops = O.ScalarOps(L, lambda u: u * u, T / m)
            errs.append(abs(O.integrate(ops, np.array(u0), m, scheme) - exact))
        slope = np.log(errs[-2] / errs[-1]) / np.log(2.0)
        assert abs(slope - order) < 0.25, (scheme, slope)


def test_grid_convergence_orders():
    """Observed orders on the 2-D 16x16 ADR problem (fixed spatial grid, T = 0.1,
    smooth datum) against a Lawson4 solution with 4096 steps."""
    dims = (16, 16)
    prob = O.ADRProblem(dims, W.sine_product_coefficient(dims), (10.0, 10.0), W.REACTION_U2_1MU)
    u0 = W.smooth_initial_state(dims, noise=0.0)
    T = 0.1
    ref = O.integrate(O.GridOps(prob, T / 4096), u0, 4096, "lawson4")
    slopes = {}
    for scheme in ("lawson_euler", "etd2rk", "lawson4"):
        e1 = O.rel_l2(O.integrate(O.GridOps(prob, T / 128), u0, 128, scheme), ref)
        e2 = O.rel_l2(O.integrate(O.GridOps(prob, T / 256), u0, 256, scheme), ref)
        slopes[scheme] = np.log(e1 / e2) / np.log(2.0)
    assert 0.8 < slopes["lawson_euler"] < 1.2, slopes
    assert 1.8 < slopes["etd2rk"] < 2.2, slopes
    assert 3.4 < slopes["lawson4"] < 4.4, slopes


# ------------------------------------------------ mixed boundary conditions, a Lap u form
def _mixed_case(dims, seed=4):
    rng = np.random.default_rng(seed)
    a = 0.5 + rng.random(tuple(n + 2 for n in dims[::-1]))
    b = (0.7, -1.3, 2.1)[: len(dims)]
    return O.ADRProblem(dims, a, b, (0.1, -0.4, 0.3, 0.2), bc="mixed", form="adelta")


@pytest.mark.parametrize("dims", [(7, 6, 5), (9, 8)])
def test_mixed_adelta_stencil_exact_for_mirror_symmetric_quadratics(dims):
    """u = prod_mu x_mu (2 - x_mu) vanishes on x_mu = 0, has zero normal derivative on x_mu = 1
    and is even about x_mu = 1, so the centred differences with the mirror ghost are exact:
    F_h u = a Lap u + b . grad u + r(u) at every node, including the Neumann ones."""
    prob = _mixed_case(dims)
    axes = [np.arange(1, n + 1) / n for n in dims]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]       # x1, x2, ...
    q = [x * (2 - x) for x in grids]
    u = np.prod(q, axis=0)
    lap = sum(-2.0 * np.prod([q[nu] for nu in range(len(dims)) if nu != mu], axis=0) for mu in range(len(dims)))
    grad = [(2 - 2 * grids[mu]) * np.prod([q[nu] for nu in range(len(dims)) if nu != mu], axis=0)
            for mu in range(len(dims))]
    a_in = prob.a[(slice(1, -1),) * len(dims)]
    exact = a_in * lap + sum(prob.b[mu] * grad[mu] for mu in range(len(dims))) + prob.reaction(u)
    assert np.max(np.abs(prob.F(u) - exact)) <= 1e-11 * np.max(np.abs(exact))


@pytest.mark.parametrize("dims", [(7, 6, 5), (9, 8)])
def test_mixed_factors_match_the_stencil_with_constant_coefficient(dims):
    """With a = a_max everywhere and r = 0, F is the constant-coefficient operator A: the
    Kronecker sum of the 1-D factors (Neumann rows included) applied densely must agree."""
    prob0 = _mixed_case(dims)
    a = np.full(prob0.a.shape, 0.8)
    prob = O.ADRProblem(dims, a, prob0.b, (0, 0, 0, 0), bc="mixed", form="adelta")
    u = np.random.default_rng(2).standard_normal(tuple(dims[::-1]))
    A = O.kron_sum_dense([prob.factor(mu) for mu in range(1, len(dims) + 1)])
    ref = (A @ u.ravel()).reshape(u.shape)
    assert np.linalg.norm(prob.F(u) - ref) <= 1e-13 * np.linalg.norm(ref)
    assert np.linalg.norm(prob.A_apply(u) - ref) <= 1e-13 * np.linalg.norm(ref)
    # and the splitting identity g = F - A u with a variable coefficient
    u2 = np.random.default_rng(3).standard_normal(tuple(dims[::-1]))
    lhs = prob0.g(u2)
    rhs = prob0.F(u2) - prob0.A_apply(u2)
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(prob0.F(u2))


def test_mixed_exp_action_matches_dense_expm():
    """e^{tau A} by mu-mode products with the (non-Toeplitz) mixed factors equals the
    dense exponential of the full Kronecker sum."""
    dims = (6, 5, 4)
    prob = _mixed_case(dims)
    tau = 3e-3
    v = np.random.default_rng(8).standard_normal(tuple(dims[::-1]))
    A = O.kron_sum_dense([prob.factor(mu) for mu in range(1, 4)])
    ref = sla.expm(tau * A) @ v.ravel()
    got = O.MatrixFunctions(prob, tau).exp_action(1.0, v).ravel()
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)


def test_e4_workload_recipe():
    """The paper's three-dimensional datum and coefficients on the mixed-BC grid."""
    from paper_2303_15861_gb300 import workloads as W
    w = W.config_e4(n=16, m=8)
    assert w.a_nodes.shape == (18, 18, 18) and w.u0.shape == (16, 16, 16)
    assert abs(w.a_nodes.max() - 0.1) < 1e-3 and w.u0.max() <= 1.0 + 1e-12
    prob = O.ADRProblem(w.dims, w.a_nodes, w.b, w.r_poly, bc="mixed", form="adelta")
    assert np.allclose(prob.beta, w.b[:3]) and prob.h[0] == 1.0 / 16


# ------------------------------------------------ periodic Fourier pseudospectral problem
def _periodic_case(dims, seed=6):
    rng = np.random.default_rng(seed)
    shape = tuple(dims[::-1])
    a = [0.4 + 0.2 * rng.random(shape) for _ in dims]
    b = [0.3 * rng.standard_normal(shape) for _ in dims]
    return a, b


@pytest.mark.parametrize("dims", [(16, 12), (8, 6, 10)])
def test_periodic_derivatives_exact_for_trigonometric_polynomials(dims):
    """Band-limited u = prod sin(2 pi p_mu x_mu / L + c_mu): D_mu and F with constant a and b
    (a Lap u + b . grad u) are exact."""
    L = 5.0
    d = len(dims)
    axes = [np.arange(n) * L / n for n in dims]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    p = [1, 2, 3][:d]
    c = [0.3, -1.1, 0.7][:d]
    f = [np.sin(2 * np.pi * p[m] * grids[m] / L + c[m]) for m in range(d)]
    fp = [2 * np.pi * p[m] / L * np.cos(2 * np.pi * p[m] * grids[m] / L + c[m]) for m in range(d)]
    fpp = [-(2 * np.pi * p[m] / L) ** 2 * f[m] for m in range(d)]
    u = np.prod(f, axis=0)
    shape = tuple(dims[::-1])
    a = [np.full(shape, 0.7), np.full(shape, 0.4), np.full(shape, 1.3)][:d]
    b = [np.full(shape, 0.9), np.full(shape, -0.5), np.full(shape, 0.2)][:d]
    prob = O.PeriodicProblem(dims, L, a, b, (0.0, 0.0, 0.0, 0.0))
    others = lambda m, g: np.prod([g[m]] + [f[q] for q in range(d) if q != m], axis=0)
    for mu in range(1, d + 1):
        assert np.abs(prob.D(u, mu) - others(mu - 1, fp)).max() < 1e-12
    exact = sum(a[m][0].flat[0] * others(m, fpp) + b[m].flat[0] * others(m, fp) for m in range(d))
    assert np.abs(prob.F(u) - exact).max() < 1e-11 * np.abs(exact).max()


@pytest.mark.parametrize("k", [0, 1, 2])
def test_periodic_matrix_functions_match_dense_exponentials(k):
    """The Fourier multipliers e^{tau s}, phi_k(tau s) against the dense augmented-matrix
    exponential of the matrix of A (assembled column by column from A_apply)."""
    dims = (8, 6)
    a, b = _periodic_case(dims)
    prob = O.PeriodicProblem(dims, 4.0, a, b, (0.0, 0.2, 0.1, 0.0), lam=0.8)
    N = 48
    A = np.stack([prob.A_apply(np.eye(N)[j].reshape(6, 8)).ravel() for j in range(N)], axis=1)
    tau = 0.05
    v = np.random.default_rng(2).standard_normal((6, 8))
    Z = np.zeros((N + 2, N + 2))
    Z[:N, :N] = tau * A
    Z[:N, N] = v.ravel()
    Z[N, N + 1] = 1.0
    big = O.expm(Z)
    ref = (O.expm(tau * A) @ v.ravel()) if k == 0 else big[:N, N + k - 1]
    ops = O.PeriodicOps(prob, tau)
    got = (ops.expA(1.0, v) if k == 0 else ops.phi(k, 1.0, v)).ravel()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_periodic_splitting_and_coefficients():
    """g = F - A u, a_max = lambda max a_mumu, beta = mean b (the d a term averages out)."""
    dims = (12, 10)
    a, b = _periodic_case(dims)
    prob = O.PeriodicProblem(dims, 3.0, a, b, (0.1, -0.3, 0.2, 0.05), lam=0.6)
    u = np.random.default_rng(1).standard_normal((10, 12))
    assert np.linalg.norm(prob.g(u) - (prob.F(u) - prob.A_apply(u))) <= 1e-12 * np.linalg.norm(prob.F(u))
    assert np.allclose(prob.amax, [0.6 * x.max() for x in a]) and np.allclose(prob.beta, [x.mean() for x in b])


def test_e3_workload_recipe():
    from paper_2303_15861_gb300 import workloads as W
    w, L, a, b = W.config_e3(n=64, m=16)
    prob = O.PeriodicProblem(w.dims, L, a, b, w.r_poly)
    assert abs(prob.amax[0] - (0.5 + 1 / 6)) < 1e-2 and abs(prob.beta[0] - 0.1) < 1e-12
    assert abs(w.u0.max() - 1.0) < 1e-12

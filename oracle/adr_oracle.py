"""FP64 oracle: semidiscrete ADR operators, exact matrix functions, integrators.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Plain numpy, FP64 throughout,
written for a reader checking it against the paper by eye; no blocking or fusion.

What it follows, function by function:
  * split_operator / ADRProblem.abar, .beta -- Eqs. (linop), (nonlin), (amaxbeta)
    of Section 3: A = lambda * sum_mu a_max d_mumu + beta . grad, with
    a_max = max a and beta_mu = |Omega|^-1 int (b_mu + d_mu a) dx.
  * ADRProblem.F / .g -- the right-hand side of Eq. (adr) and the remainder
    g = F - A u of Eq. (nonlin), discretised with second-order centred finite
    differences (Section 5.2), conservative flux form, Dirichlet ghosts = 0.
  * factor -- the 1-D factor A_mu of the Kronecker sum A_3 (+) A_2 (+) A_1
    (Section 5.2).
  * expm -- scaling and squaring with the [13/13] Pade approximant
    (Higham 2005, the method the paper's mu-mode code relies on via expm).
  * apply_mode / exp_action -- the mu-mode (Tucker) identity
    exp(A_d (+) ... (+) A_1) v = vec(V x_1 e^{A_1} ... x_d e^{A_d}) (Section 1).
  * phi -- phi_1(z) = (e^z - 1)/z, phi_2(z) = (phi_1(z) - 1)/z (Section 1,
    Theorem 2.4), removable singularity handled by the Taylor series.
  * phi_action -- phi_k of the Kronecker sum through the joint eigenbasis of the
    1-D factors (numpy.linalg.eig), the pointwise phi_k(tau*(l1+l2+l3)) scaling,
    and the back transform.
  * step_* -- the integrators of the Appendix (Lawson type, classical
    exponential), plus Lawson4: Lawson's construction (Section 1) applied to the
    classical fourth-order Runge--Kutta method.

Readings where the paper is silent:
  * face coefficient a_{i+1/2} = (a_i + a_{i+1}) / 2 of the nodal a (incl. boundary);
  * a_max is the maximum over the nodal samples unless an override is given;
  * beta_mu = b_mu + mean over the two boundary faces x_mu = 0, 1 of the jump of a
    (trapezoidal weights), i.e. Eq. (amaxbeta) with the exact integral of d_mu a;
  * phi_k near zero: Taylor series for |z| < 1, closed forms elsewhere.
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial

import numpy as np

# ----------------------------------------------------------------------------------
# phi functions (Section 1 and Theorem 2.4)
# ----------------------------------------------------------------------------------


def phi(k: int, z):
    """phi_0 = exp, phi_1(z) = (e^z-1)/z, phi_2(z) = (phi_1(z)-1)/z, elementwise FP64.

    For |z| < 1 the Taylor series sum_j z^j / (j+k)! is summed to FP64 accuracy,
    which avoids the cancellation of the closed forms near the removable singularity.
    """
    z = np.asarray(z, dtype=np.float64)
    if k == 0:
        return np.exp(z)
    out = np.empty_like(z)
    small = np.abs(z) < 1.0
    zs = z[small]
    acc = np.zeros_like(zs)
    term = np.full_like(zs, 1.0 / factorial(k))
    for j in range(0, 30):                      # |z|<1: 30 terms is far below 1e-17
        acc = acc + term
        term = term * zs / (j + k + 1)
    out[small] = acc
    zl = z[~small]
    if k == 1:
        out[~small] = np.expm1(zl) / zl
    elif k == 2:
        out[~small] = (np.expm1(zl) - zl) / (zl * zl)
    else:
        raise ValueError("phi_k implemented for k <= 2")
    return out


# ----------------------------------------------------------------------------------
# Matrix exponential: scaling and squaring with the [13/13] Pade approximant
# ----------------------------------------------------------------------------------

def _pade_exp_coefficients(m: int):
    """Coefficients of the numerator of the [m/m] Pade approximant to e^x:
    c_j = (2m-j)! m! / ((2m)! j! (m-j)!)."""
    return [float(Fraction(factorial(2 * m - j) * factorial(m),
                           factorial(2 * m) * factorial(j) * factorial(m - j)))
            for j in range(m + 1)]


_PADE13 = _pade_exp_coefficients(13)
THETA13 = 5.371920351148152   # 1-norm bound for degree 13 (Higham 2005, Table 2.3)


def expm(A: np.ndarray) -> np.ndarray:
    """exp(A) by scaling and squaring with the [13/13] Pade approximant."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    nrm = np.linalg.norm(A, 1)
    s = 0
    if nrm > THETA13:
        s = int(np.ceil(np.log2(nrm / THETA13)))
    As = A / (2.0 ** s)
    c = _PADE13
    I = np.eye(n)
    A2 = As @ As
    A4 = A2 @ A2
    A6 = A4 @ A2
    U = As @ (A6 @ (c[13] * A6 + c[11] * A4 + c[9] * A2)
              + c[7] * A6 + c[5] * A4 + c[3] * A2 + c[1] * I)
    V = (A6 @ (c[12] * A6 + c[10] * A4 + c[8] * A2)
         + c[6] * A6 + c[4] * A4 + c[2] * A2 + c[0] * I)
    R = np.linalg.solve(V - U, V + U)
    for _ in range(s):
        R = R @ R
    return R


# ----------------------------------------------------------------------------------
# mu-mode products (Section 1, Section 5.2)
# ----------------------------------------------------------------------------------

def apply_mode(U: np.ndarray, M: np.ndarray, mu: int) -> np.ndarray:
    """U x_mu M: contract direction mu (1 = x1, the fastest numpy axis) with M."""
    ax = U.ndim - mu
    return np.moveaxis(np.tensordot(M, U, axes=([1], [ax])), 0, ax)


def kron_sum_dense(factors) -> np.ndarray:
    """Dense A_d (+) ... (+) A_1 acting on vec(U) with x1 fastest (tiny grids only)."""
    d = len(factors)
    ns = [f.shape[0] for f in factors]
    total = int(np.prod(ns))
    out = np.zeros((total, total))
    for mu in range(1, d + 1):
        term = np.ones((1, 1))
        for nu in range(d, 0, -1):          # slowest direction first in the product
            term = np.kron(term, factors[mu - 1] if nu == mu else np.eye(ns[nu - 1]))
        out += term
    return out


# ----------------------------------------------------------------------------------
# The problem: operator extraction and finite-difference stencils (Sections 3, 5.2)
# ----------------------------------------------------------------------------------

class ADRProblem:
    """u_t = div(a grad u) + b . grad u + r(u) on (0,1)^d, homogeneous Dirichlet (form
    "flux", bc "dirichlet"); or, as in the paper's three-dimensional experiment (Section 5.2,
    Eq. (adr3d)), u_t = a Lap u + b . grad u + r(u) (form "adelta") with homogeneous Dirichlet
    values on the faces x_mu = 0 and homogeneous Neumann values on the faces x_mu = 1
    (bc "mixed"; only with form "adelta").

    dims: unknowns per direction, x1 first. Dirichlet: nodes x_i = i h, h = 1/(n+1),
    i = 1..n. Mixed: h = 1/n, i = 1..n (x_n = 1 is an unknown; the Neumann condition enters
    through the mirror ghost u_{n+1} = u_{n-1}). a_nodes: nodal a at x_j = j h, j = 0..n+1,
    numpy shape (n_d+2, ..., n_1+2). b: constant velocity (length >= d).
    r_poly: r(u) = r0 + r1 u + r2 u^2 + r3 u^3. lam: the lambda of Eq. (linop).
    """

    def __init__(self, dims, a_nodes, b, r_poly, lam=1.0, abar=None, bc="dirichlet", form="flux"):
        self.dims = tuple(int(n) for n in dims)
        self.d = len(self.dims)
        self.a = np.asarray(a_nodes, dtype=np.float64)
        assert self.a.shape == tuple(n + 2 for n in self.dims[::-1])
        assert bc in ("dirichlet", "mixed") and form in ("flux", "adelta")
        assert bc == "dirichlet" or form == "adelta", "Neumann faces are supported for the a Lap u form"
        self.bc, self.form = bc, form
        self.b = np.asarray(b, dtype=np.float64)[: self.d]
        self.r = tuple(float(c) for c in r_poly)
        self.lam = float(lam)
        self.h = [1.0 / (n + 1) if bc == "dirichlet" else 1.0 / n for n in self.dims]
        # Eq. (amaxbeta): a_max = max a over the nodes of the closed domain (unless overridden)
        dom = self.a if bc == "dirichlet" else self.a[tuple(slice(0, n + 1) for n in self.dims[::-1])]
        self.abar = self.lam * float(dom.max()) if abar is None else float(abar)
        if form == "flux":
            self.beta = np.array([self.b[mu - 1] + self._mean_face_jump(mu) for mu in range(1, self.d + 1)])
        else:   # a Lap u: A = lambda a_max Lap + b . grad (Eq. (adr3dstab))
            self.beta = self.b.copy()

    # -- Eq. (amaxbeta): the domain mean of d_mu a is the face-mean of a(x_mu=1)-a(x_mu=0)
    def _mean_face_jump(self, mu):
        ax = self.d - mu
        hi = np.take(self.a, -1, axis=ax)
        lo = np.take(self.a, 0, axis=ax)
        return float(self._trapz_mean(hi - lo))

    @staticmethod
    def _trapz_mean(f):
        """Mean over the unit (d-1)-cube of nodal values, trapezoidal weights."""
        f = np.asarray(f, dtype=np.float64)
        while f.ndim > 0:
            m = f.shape[0]
            w = np.ones(m)
            w[0] = w[-1] = 0.5
            f = np.tensordot(w / (m - 1), f, axes=([0], [0]))
        return f

    # -- reaction
    def reaction(self, u):
        r0, r1, r2, r3 = self.r
        return r0 + u * (r1 + u * (r2 + u * r3))

    # -- stencil with a face coefficient field and velocity
    def _flux_form(self, u, coef, vel):
        d = self.d
        up = np.pad(u, 1)                       # Dirichlet: ghost values are zero
        out = np.zeros_like(u)
        inner = (slice(1, -1),) * d
        for mu in range(1, d + 1):
            ax = d - mu
            h = self.h[mu - 1]
            plus = list(inner)
            minus = list(inner)
            plus[ax] = slice(2, None)
            minus[ax] = slice(0, -2)
            plus, minus = tuple(plus), tuple(minus)
            uc, up_, um = up[inner], up[plus], up[minus]
            ac, ap, am = coef[inner], coef[plus], coef[minus]
            a_plus = 0.5 * (ac + ap)            # face coefficient a_{i+1/2}
            a_minus = 0.5 * (ac + am)           # face coefficient a_{i-1/2}
            out += (a_plus * (up_ - uc) - a_minus * (uc - um)) / (h * h)
            out += vel[mu - 1] * (up_ - um) / (2.0 * h)
        return out

    # -- a Lap u + vel . grad u with the ghost values of the boundary conditions
    def _padded(self, u):
        up = np.pad(u, 1)                       # Dirichlet ghosts: zero
        if self.bc == "mixed":                  # Neumann on x_mu = 1: u_{n+1} = u_{n-1}
            for ax in range(self.d):
                hi = [slice(None)] * self.d
                src = [slice(None)] * self.d
                hi[ax] = -1
                src[ax] = -3
                up[tuple(hi)] = up[tuple(src)]
        return up

    def _adelta_form(self, u, coef, vel):
        d = self.d
        up = self._padded(u)
        inner = (slice(1, -1),) * d
        lap = np.zeros_like(u)
        adv = np.zeros_like(u)
        for mu in range(1, d + 1):
            ax = d - mu
            h = self.h[mu - 1]
            plus = list(inner)
            minus = list(inner)
            plus[ax] = slice(2, None)
            minus[ax] = slice(0, -2)
            uc, upl, umi = up[inner], up[tuple(plus)], up[tuple(minus)]
            lap += (upl - 2.0 * uc + umi) / (h * h)
            adv += vel[mu - 1] * (upl - umi) / (2.0 * h)
        return coef[inner] * lap + adv

    def F(self, u):
        """Full semidiscrete right-hand side of Eq. (adr) (or Eq. (adr3d) for form "adelta")."""
        if self.form == "adelta":
            return self._adelta_form(u, self.a, self.b) + self.reaction(u)
        return self._flux_form(u, self.a, self.b) + self.reaction(u)

    def g(self, u):
        """Remainder of Eq. (nonlin), written directly with (a - a_max) and (b - beta)."""
        if self.form == "adelta":
            return self._adelta_form(u, self.a - self.abar, self.b - self.beta) + self.reaction(u)
        return self._flux_form(u, self.a - self.abar, self.b - self.beta) + self.reaction(u)

    # -- 1-D factors of the Kronecker sum (Section 5.2)
    def factor(self, mu):
        """A_mu: tridiagonal discretisation of a_max d_mumu + beta_mu d_mu."""
        n = self.dims[mu - 1]
        h = self.h[mu - 1]
        diag = -2.0 * self.abar / (h * h)
        sup = self.abar / (h * h) + self.beta[mu - 1] / (2.0 * h)   # coefficient of u_{i+1}
        sub = self.abar / (h * h) - self.beta[mu - 1] / (2.0 * h)   # coefficient of u_{i-1}
        A = (np.diag(np.full(n, diag)) + np.diag(np.full(n - 1, sup), 1)
             + np.diag(np.full(n - 1, sub), -1))
        if self.bc == "mixed":
            # last node: the mirror ghost u_{n+1} = u_{n-1} turns its row into
            # a_max (2 u_{n-1} - 2 u_n) / h^2 and cancels the central advection
            A[n - 1, n - 2] = 2.0 * self.abar / (h * h)
        return A

    def A_apply(self, u):
        """A u through the Kronecker-sum factors: sum_mu U x_mu A_mu."""
        out = np.zeros_like(u)
        for mu in range(1, self.d + 1):
            out += apply_mode(u, self.factor(mu), mu)
        return out


class MatrixFunctions:
    """Exact (to FP64 rounding) actions of e^{c tau A} and phi_k(c tau A)."""

    def __init__(self, prob: ADRProblem, tau: float):
        self.p = prob
        self.tau = float(tau)
        self._E = {}
        self._eig = None

    def E_factors(self, c):
        key = float(c)
        if key not in self._E:
            self._E[key] = [expm(c * self.tau * self.p.factor(mu)) for mu in range(1, self.p.d + 1)]
        return self._E[key]

    def exp_action(self, c, v):
        """e^{c tau A} v = V x_1 e^{c tau A_1} x_2 ... x_d e^{c tau A_d} (Section 1)."""
        out = v
        for mu, E in enumerate(self.E_factors(c), start=1):
            out = apply_mode(out, E, mu)
        return out

    def eig(self):
        if self._eig is None:
            res = []
            for mu in range(1, self.p.d + 1):
                w, V = np.linalg.eig(self.p.factor(mu))
                if np.max(np.abs(np.imag(w))) > 0 or np.max(np.abs(np.imag(V))) > 0:
                    raise ValueError("complex spectrum: the eigen route needs real eigenvalues")
                w = np.real(w)
                V = np.real(V)
                res.append((w, V, np.linalg.inv(V)))
            self._eig = res
        return self._eig

    def phi_action_dense(self, k, c, v):
        """phi_k(c tau A) v for any conditioning of the eigenbasis (small grids only): the
        exponential of the augmented matrix Z = [[c tau A, v, 0], [0, 0, 1], [0, 0, 0]] holds
        e^{c tau A} v, phi_1(c tau A) v and phi_2(c tau A) v in its last columns, with A the
        full Kronecker sum A_d (+) ... (+) A_1 (Section 5.2), formed densely."""
        A = kron_sum_dense([self.p.factor(mu) for mu in range(1, self.p.d + 1)])
        N = v.size
        Z = np.zeros((N + 2, N + 2))
        Z[:N, :N] = c * self.tau * A
        Z[:N, N] = np.ravel(v)
        Z[N, N + 1] = 1.0
        big = expm(Z)
        col = {0: None, 1: N, 2: N + 1}[k]
        if col is None:
            return (expm(c * self.tau * A) @ np.ravel(v)).reshape(v.shape)
        return big[:N, col].reshape(v.shape)

    def phi_action(self, k, c, v):
        """phi_k(c tau A) v through the joint eigenbasis of the 1-D factors."""
        eig = self.eig()
        out = v
        for mu, (w, V, Vi) in enumerate(eig, start=1):
            out = apply_mode(out, Vi, mu)
        lam_sum = np.zeros(v.shape)
        for mu, (w, V, Vi) in enumerate(eig, start=1):
            shape = [1] * v.ndim
            shape[v.ndim - mu] = w.size
            lam_sum = lam_sum + w.reshape(shape)
        out = out * phi(k, c * self.tau * lam_sum)
        for mu, (w, V, Vi) in enumerate(eig, start=1):
            out = apply_mode(out, V, mu)
        return out


def phi_complex(k: int, z):
    """phi_k of complex arguments (elementwise, FP64): the Taylor series for |z| < 1,
    the closed forms e^z, (e^z - 1)/z, (e^z - 1 - z)/z^2 elsewhere."""
    z = np.asarray(z, dtype=np.complex128)
    if k == 0:
        return np.exp(z)
    out = np.empty_like(z)
    small = np.abs(z) < 1.0
    zs = z[small]
    acc = np.zeros_like(zs)
    term = np.full_like(zs, 1.0 / factorial(k))
    for j in range(0, 30):
        acc = acc + term
        term = term * zs / (j + k + 1)
    out[small] = acc
    zl = z[~small]
    e = np.expm1(zl.real) * np.exp(1j * zl.imag) + (np.exp(1j * zl.imag) - 1.0)   # e^z - 1
    out[~small] = e / zl if k == 1 else (e - zl) / (zl * zl)
    return out


class PeriodicProblem:
    """The paper's two-dimensional experiment form (Section 5.1, Eq. (ad2d)):
    u_t = div(a grad u) + div(b u) + r(u) on a periodic box of side L, with a diagonal
    diffusion tensor a = diag(a_11, ..., a_dd) and a velocity field b(x), both sampled at the
    nodes x_j = x0 + j L/n, discretised by the Fourier pseudospectral method (n modes per
    direction; first derivatives D_mu with the Nyquist wavenumber set to zero).

    A of Eq. (linop) = lambda sum_mu a_mumu^max D_mu^2 + beta . D with a_mumu^max the nodal
    maximum and beta_mu the mean of b_mu (Eq. (amaxbeta); d_mu a_mumu averages to zero over a
    period). A is diagonal in Fourier space with symbol
    s(k) = -lambda sum_mu a^max_mu k_mu^2 + i beta . k.
    a_diag, b_field: d nodal arrays each, numpy shape (n_d, ..., n_1)."""

    def __init__(self, dims, L, a_diag, b_field, r_poly, lam=1.0, form="flux"):
        if form not in ("flux", "adelta"):
            raise ValueError("form must be 'flux' or 'adelta'")
        self.form = form
        self.dims = tuple(int(n) for n in dims)
        self.d = len(self.dims)
        self.L = float(L)
        shape = self.dims[::-1]
        self.a = [np.asarray(x, dtype=np.float64).reshape(shape) for x in a_diag]
        self.bf = [np.asarray(x, dtype=np.float64).reshape(shape) for x in b_field]
        self.r = tuple(float(c) for c in r_poly)
        self.lam = float(lam)
        self.amax = np.array([self.lam * float(x.max()) for x in self.a])
        self.beta = np.array([float(x.mean()) for x in self.bf])
        self.k = []
        for mu in range(1, self.d + 1):
            n = self.dims[mu - 1]
            km = np.fft.fftfreq(n, d=1.0 / n) * (2.0 * np.pi / self.L)
            if n % 2 == 0:
                km[n // 2] = 0.0                      # Nyquist: no first derivative
            shp = [1] * self.d
            shp[self.d - mu] = n
            self.k.append(km.reshape(shp))
        self.symbol = sum(-self.amax[mu] * self.k[mu] ** 2 + 1j * self.beta[mu] * self.k[mu]
                          for mu in range(self.d))

    def D(self, u, mu):
        """Pseudospectral first derivative along x_mu (mu = 1..d)."""
        return np.real(np.fft.ifftn(1j * self.k[mu - 1] * np.fft.fftn(u)))

    def reaction(self, u):
        r0, r1, r2, r3 = self.r
        return r0 + u * (r1 + u * (r2 + u * r3))

    def F(self, u):
        """sum_mu D_mu (a_mumu D_mu u + b_mu u) + r(u); for form "adelta" (the one-dimensional
        linear experiment of Section 4, Eq. (adlinearzero)) sum_mu (a_mumu D_mu D_mu u + D_mu (b_mu u)) + r(u)."""
        if self.form == "adelta":
            return sum(self.a[mu - 1] * self.D(self.D(u, mu), mu) + self.D(self.bf[mu - 1] * u, mu)
                       for mu in range(1, self.d + 1)) + self.reaction(u)
        return sum(self.D(self.a[mu - 1] * self.D(u, mu) + self.bf[mu - 1] * u, mu)
                   for mu in range(1, self.d + 1)) + self.reaction(u)

    def g(self, u):
        """Eq. (nonlin): sum_mu D_mu ((a_mumu - lambda a^max) D_mu u + (b_mu - beta_mu) u) + r(u);
        for form "adelta" (Eq. (ex0stab)) (a_mumu - lambda a^max) D_mu D_mu u in place of the flux."""
        if self.form == "adelta":
            return sum((self.a[mu - 1] - self.amax[mu - 1]) * self.D(self.D(u, mu), mu)
                       + self.D((self.bf[mu - 1] - self.beta[mu - 1]) * u, mu)
                       for mu in range(1, self.d + 1)) + self.reaction(u)
        return sum(self.D((self.a[mu - 1] - self.amax[mu - 1]) * self.D(u, mu)
                          + (self.bf[mu - 1] - self.beta[mu - 1]) * u, mu)
                   for mu in range(1, self.d + 1)) + self.reaction(u)

    def A_apply(self, u):
        return np.real(np.fft.ifftn(self.symbol * np.fft.fftn(u)))


def periodic_linear_exact(prob: PeriodicProblem, u0, T):
    """The exact solution exp(T M) u0 of the semidiscrete problem u' = M u = F(u) for a
    one-dimensional "adelta" problem without advection and reaction (the linear experiment of
    Section 4, Eq. (adlinearzero)): M = diag(a) D D with D the pseudospectral derivative, which is
    similar to the symmetric diag(a)^{1/2} D D diag(a)^{1/2}; its eigendecomposition gives the
    exponential. Dense, so for n up to a few thousand."""
    if prob.d != 1 or prob.form != "adelta" or any(c != 0.0 for c in prob.r) or np.any(prob.bf[0] != 0.0):
        raise ValueError("only the 1-D a u_xx problem without advection or reaction")
    n = prob.dims[0]
    eye = np.eye(n)
    D2 = np.real(np.fft.ifft((1j * prob.k[0].reshape(-1, 1)) ** 2 * np.fft.fft(eye, axis=0), axis=0))
    D2 = 0.5 * (D2 + D2.T)                       # symmetric up to rounding
    sa = np.sqrt(prob.a[0])
    w, V = np.linalg.eigh(sa[:, None] * D2 * sa[None, :])
    u0 = np.asarray(u0, dtype=np.float64)
    return sa * (V @ (np.exp(T * w) * (V.T @ (u0 / sa))))


class PeriodicOps:
    """The operations every integrator needs, for the periodic pseudospectral problem: the
    matrix functions of A are pointwise multipliers on the Fourier coefficients."""

    def __init__(self, prob: PeriodicProblem, tau: float):
        self.prob = prob
        self.tau = float(tau)
        self._mult = {}                       # the multipliers already formed, by (k, c)

    def g(self, u):
        return self.prob.g(u)

    def F(self, u):
        return self.prob.F(u)

    def _multiplier(self, k, c):
        key = (k, float(c))
        if key not in self._mult:
            z = c * self.tau * self.prob.symbol
            self._mult[key] = np.exp(z) if k == 0 else phi_complex(k, z)
        return self._mult[key]

    def expA(self, c, v):
        return np.real(np.fft.ifftn(self._multiplier(0, c) * np.fft.fftn(v)))

    def phi(self, k, c, v):
        return np.real(np.fft.ifftn(self._multiplier(k, c) * np.fft.fftn(v)))


def solve_periodic(dims, L, a_diag, b_field, r_poly, u0, tau, m, scheme, lam=1.0, form="flux"):
    """FP64 oracle solution of the periodic problem after m steps of `scheme`."""
    prob = PeriodicProblem(dims, L, a_diag, b_field, r_poly, lam=lam, form=form)
    return integrate(PeriodicOps(prob, tau), u0, m, scheme)


class GridOps:
    """The operations every integrator needs, for an ADR grid problem. phi_route "eigen"
    (the joint eigenbasis) or "dense" (the augmented-matrix exponential, small grids, any
    conditioning of the eigenbasis)."""

    def __init__(self, prob: ADRProblem, tau: float, phi_route: str = "eigen"):
        self.prob = prob
        self.tau = float(tau)
        self.mf = MatrixFunctions(prob, tau)
        self.phi_route = phi_route

    def g(self, u):
        return self.prob.g(u)

    def F(self, u):
        return self.prob.F(u)

    def expA(self, c, v):
        return self.mf.exp_action(c, v)

    def phi(self, k, c, v):
        if self.phi_route == "dense":
            return self.mf.phi_action_dense(k, c, v)
        return self.mf.phi_action(k, c, v)


class ScalarOps:
    """u' = A u + g(u) for a scalar (or elementwise array) linear part A and callable g.

    Used by the stability-function and scalar-convergence pins: with A = lam z and
    g(u) = (1-lam) z u one step from u = 1 gives the stability function Phi(z, lam).
    """

    def __init__(self, A, g, tau):
        self.A = np.asarray(A, dtype=np.float64)
        self._g = g
        self.tau = float(tau)

    def g(self, u):
        return self._g(u)

    def F(self, u):
        return self.A * u + self._g(u)

    def expA(self, c, v):
        return np.exp(c * self.tau * self.A) * v

    def phi(self, k, c, v):
        return phi(k, c * self.tau * self.A) * v


# ----------------------------------------------------------------------------------
# Integrators (Appendix; Lawson4 derived from Lawson's construction)
# ----------------------------------------------------------------------------------

def step_lawson_euler(ops, u):
    """u+ = e^{tau A}(u + tau g(u))."""
    return ops.expA(1.0, u + ops.tau * ops.g(u))


def step_stabilized_lawson_euler(ops, u):
    """u+ = u + tau e^{tau A} F(u)."""
    return u + ops.tau * ops.expA(1.0, ops.F(u))


def step_lawson2a(ops, u):
    t = ops.tau
    U = ops.expA(0.5, u + 0.5 * t * ops.g(u))
    return ops.expA(1.0, u) + t * ops.expA(0.5, ops.g(U))


def step_lawson2b(ops, u):
    t = ops.tau
    gu = ops.g(u)
    U = ops.expA(1.0, u + t * gu)
    return ops.expA(1.0, u + 0.5 * t * gu) + 0.5 * t * ops.g(U)


def step_stabilized_lawson2(ops, u, alpha=0.327):
    t = ops.tau
    Fu = ops.F(u)
    U = u + alpha * t * ops.expA(alpha, Fu)
    return (u + t * ops.expA(0.5, Fu)
            + t / (2.0 * alpha) * ops.expA(1.0, ops.g(U) - ops.g(u)))


def step_exponential_euler(ops, u):
    """u+ = u + tau phi_1(tau A) F(u)."""
    return u + ops.tau * ops.phi(1, 1.0, ops.F(u))


def step_erk2p2(ops, u, c2=1.0):
    """Exponential Runge--Kutta, second order, with phi_2 (Appendix)."""
    t = ops.tau
    Fu = ops.F(u)
    U = u + c2 * t * ops.phi(1, c2, Fu)
    return (u + t * ops.phi(1, 1.0, Fu)
            + t / c2 * ops.phi(2, 1.0, ops.g(U) - ops.g(u)))


def step_erk2p1(ops, u, c2=1.0):
    """Exponential Runge--Kutta, second order, phi_1 only (Appendix)."""
    t = ops.tau
    Fu = ops.F(u)
    U = u + c2 * t * ops.phi(1, c2, Fu)
    return (u + t * ops.phi(1, 1.0, Fu)
            + t / (2.0 * c2) * ops.phi(1, 1.0, ops.g(U) - ops.g(u)))


def step_lawson4(ops, u):
    """Classical RK4 applied to v = e^{-(t-t_n)A} u, written back in u (E = e^{tau A/2}):
    k1 = g(u);  U2 = E(u + tau/2 k1);  k2 = g(U2);  U3 = E u + tau/2 k2;  k3 = g(U3);
    U4 = E(E u + tau k3);  k4 = g(U4);
    u+ = E(E(u + tau/6 k1) + tau/3 (k2 + k3)) + tau/6 k4."""
    t = ops.tau
    E = lambda v: ops.expA(0.5, v)
    k1 = ops.g(u)
    U2 = E(u + 0.5 * t * k1)
    k2 = ops.g(U2)
    Eu = E(u)
    U3 = Eu + 0.5 * t * k2
    k3 = ops.g(U3)
    U4 = E(Eu + t * k3)
    k4 = ops.g(U4)
    return E(E(u + t / 6.0 * k1) + t / 3.0 * (k2 + k3)) + t / 6.0 * k4


SCHEMES = {
    "lawson_euler": step_lawson_euler,
    "etd2rk": step_erk2p2,               # erk2p2 with c2 = 1 (Cox--Matthews ETD2RK)
    "lawson4": step_lawson4,
    "exponential_euler": step_exponential_euler,
    "erk2p1": step_erk2p1,
    "stabilized_lawson_euler": step_stabilized_lawson_euler,
    "lawson2a": step_lawson2a,
    "lawson2b": step_lawson2b,
    "stabilized_lawson2": step_stabilized_lawson2,
}


def integrate(ops, u0, m, scheme):
    step = SCHEMES[scheme]
    u = np.array(u0, dtype=np.float64, copy=True)
    for _ in range(int(m)):
        u = step(ops, u)
    return u


def solve(dims, a_nodes, b, r_poly, u0, tau, m, scheme, lam=1.0, abar=None, phi_route="eigen",
          bc="dirichlet", form="flux"):
    """Convenience: FP64 oracle solution after m steps of `scheme`."""
    prob = ADRProblem(dims, a_nodes, b, r_poly, lam=lam, abar=abar, bc=bc, form=form)
    return integrate(GridOps(prob, tau, phi_route=phi_route), u0, m, scheme)


# ----------------------------------------------------------------------------------
# Error norms (relative l2 as the parity measure; relative max-norm as in the paper)
# ----------------------------------------------------------------------------------

def rel_l2(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))


def rel_inf(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))

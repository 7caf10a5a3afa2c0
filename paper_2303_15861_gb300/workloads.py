"""Seeded synthetic inputs for the advection-diffusion-reaction workloads.

This module only samples coefficient fields and initial data on the grid; it holds
none of the method's arithmetic (no stencil, no matrix function, no time stepping).
It is the one module that both the CUDA path's callers and the FP64 oracle's
callers use, so that both sides see bit-identical inputs.

Grid convention (Section 5.2 of the paper: second-order centred finite differences on
a tensor grid): the unit box (0,1)^d holds n_mu interior nodes per direction,
x_i = i*h_mu with h_mu = 1/(n_mu+1), i = 1..n_mu, and homogeneous Dirichlet values
on the boundary. Arrays are C-ordered with x1 varying fastest: a 3-D state has
numpy shape (n3, n2, n1); the nodal coefficient a(x) includes the boundary ring and
has shape (n3+2, n2+2, n1+2).

Workload recipes (stated once, used by tests and bench.py):
  * a(x) = 1 + c * prod_mu sin(2*pi*k*x_mu)       (c = 0.5, k = 1 unless batched)
  * b constant, reaction r(u) = u^2 (1 - u)        (coefficients r0..r3 = 0, 0, 1, -1)
  * 2-D u0 = 16 x(1-x) y(1-y) + 1e-3 N(0,1)
  * 3-D u0 = (27/4)^3 x1 x2 x3 (1-x1)^2 (1-x2)^2 (1-x3)^2 + 1e-3 N(0,1)
    (the smooth datum of the paper's three-dimensional experiment, Section 5.2)
  * noise from numpy.random.default_rng(seed) on interior nodes only.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

REACTION_U2_1MU = (0.0, 0.0, 1.0, -1.0)  # r(u) = u^2 - u^3


@dataclass
class Workload:
    """One ADR instance: grid, coefficients, initial state and time grid."""
    name: str
    dims: tuple            # interior points per direction, x1 first: (n1, n2[, n3])
    a_nodes: np.ndarray    # nodal diffusion coefficient incl. boundary ring, C-order
    b: tuple               # constant advection velocity (b1, b2, b3); unused entries 0
    r_poly: tuple          # reaction r(u) = r0 + r1 u + r2 u^2 + r3 u^3
    u0: np.ndarray         # initial state on interior nodes, C-order, x1 fastest
    tau: float             # time step
    m: int                 # number of steps
    scheme: str            # "lawson_euler" | "etd2rk" | "lawson4"
    extra: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return len(self.dims)

    @property
    def dof(self) -> int:
        return int(np.prod(self.dims))


def axis_nodes(n: int, with_boundary: bool) -> np.ndarray:
    """Node coordinates along one direction of the unit interval."""
    h = 1.0 / (n + 1)
    if with_boundary:
        return np.arange(0, n + 2, dtype=np.float64) * h
    return np.arange(1, n + 1, dtype=np.float64) * h


def mesh(dims, with_boundary):
    axes = [axis_nodes(n, with_boundary) for n in dims]      # x1, x2, ...
    # numpy index order is (x_d, ..., x_1) so that x1 is the fastest index
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return grids[::-1]                                        # return x1, x2, ...


def sine_product_coefficient(dims, c=0.5, k=1) -> np.ndarray:
    """a(x) = 1 + c prod_mu sin(2 pi k x_mu) sampled on all nodes incl. the boundary."""
    xs = mesh(dims, True)
    prod = np.ones_like(xs[0])
    for x in xs:
        prod = prod * np.sin(2.0 * np.pi * k * x)
    return 1.0 + c * prod


def smooth_initial_state(dims, noise=1e-3, seed=0, rng=None) -> np.ndarray:
    """Smooth datum vanishing on the boundary plus seeded Gaussian noise."""
    xs = mesh(dims, False)
    if len(dims) == 2:
        x, y = xs
        u = 16.0 * x * (1.0 - x) * y * (1.0 - y)
    else:
        u = np.full_like(xs[0], (27.0 / 4.0) ** 3)
        for x in xs:
            u = u * x * (1.0 - x) ** 2
    if noise:
        rng = np.random.default_rng(seed) if rng is None else rng
        u = u + noise * rng.standard_normal(u.shape)
    return np.ascontiguousarray(u)


def single_grid(name, dims, b, scheme, T, m, c=0.5, k=1, noise=1e-3, seed=0) -> Workload:
    dims = tuple(int(n) for n in dims)
    bb = tuple(float(v) for v in b) + (0.0,) * (3 - len(b))
    return Workload(name=name, dims=dims, a_nodes=sine_product_coefficient(dims, c, k),
                    b=bb, r_poly=REACTION_U2_1MU,
                    u0=smooth_initial_state(dims, noise=noise, seed=seed),
                    tau=T / m, m=int(m), scheme=scheme)


# --- the five workload recipes ------------------------------------------------------

def config1(scheme="etd2rk", n=32):
    """2-D 32x32, b=(10,10), 20 steps to T=0.1, FP64."""
    return single_grid(f"2d_{n}_{scheme}", (n, n), (10.0, 10.0), scheme, 0.1, 20)


def config2(n=128, m=50, scheme="etd2rk"):
    """3-D 128^3, b=(10,10,10), ETD2RK, 50 steps to T=0.1, FP64."""
    return single_grid(f"3d_{n}_{scheme}", (n, n, n), (10.0, 10.0, 10.0), scheme, 0.1 * m / 50, m)


def config3(n=256, m=40, scheme="lawson4"):
    """3-D 256^3, Lawson4, 40 steps to T=0.1 (tau = 2.5e-3), mixed precision."""
    return single_grid(f"3d_{n}_{scheme}", (n, n, n), (10.0, 10.0, 10.0), scheme, 0.1 * m / 40, m)


def config5(n=384, m=200, scheme="lawson4"):
    """3-D 384^3, b=(50,50,50), 200 steps to T=1.0."""
    return single_grid(f"3d_{n}_{scheme}_b50", (n, n, n), (50.0, 50.0, 50.0), scheme, 1.0 * m / 200, m)


BATCH_SIZES = (48, 64, 96, 128, 192, 256)


def config4_draws(count=512, seed=2303):
    """Per-instance draws of the batched 2-D workload, in a fixed order:
    n_i from BATCH_SIZES, c_i ~ U[0.1, 0.9], k_i in {1,2,3}, b_i ~ U[0,20]^2."""
    rng = np.random.default_rng(seed)
    n = rng.choice(np.array(BATCH_SIZES), size=count)
    c = rng.uniform(0.1, 0.9, size=count)
    k = rng.integers(1, 4, size=count)
    b = rng.uniform(0.0, 20.0, size=(count, 2))
    return [dict(n=int(n[i]), c=float(c[i]), k=int(k[i]), b=(float(b[i, 0]), float(b[i, 1])))
            for i in range(count)]


def config4(count=512, m=30, T=0.1, seed=2303, select=None):
    """Batched 2-D: independent instances of uneven size, ETD2RK, FP32 state. `select` (a range
    of instance indices) builds only those instances of the count-instance draw; instance i is
    the same whichever others are built."""
    out = []
    draws = config4_draws(count, seed)
    for i in (range(count) if select is None else select):
        d = draws[i]
        dims = (d["n"], d["n"])
        out.append(Workload(
            name=f"batch{i}_{d['n']}", dims=dims,
            a_nodes=sine_product_coefficient(dims, d["c"], d["k"]),
            b=(d["b"][0], d["b"][1], 0.0), r_poly=REACTION_U2_1MU,
            u0=smooth_initial_state(dims, noise=1e-3, rng=np.random.default_rng((seed, i))),
            tau=T / m, m=m, scheme="etd2rk", extra=d))
    return out


def batch_instances(sizes, m=30, T=0.1, scheme="etd2rk", seed=2303):
    """Independent 2-D instances with the given (n1, n2), each drawn like the batched
    workload above: c ~ U[0.1, 0.9], k in {1, 2, 3}, b ~ U[0, 20]^2, reaction u^2(1-u)."""
    rng = np.random.default_rng(seed)
    out = []
    for i, (n1, n2) in enumerate(sizes):
        c = float(rng.uniform(0.1, 0.9))
        k = int(rng.integers(1, 4))
        b = rng.uniform(0.0, 20.0, size=2)
        dims = (int(n1), int(n2))
        out.append(Workload(
            name=f"inst{i}_{n1}x{n2}", dims=dims,
            a_nodes=sine_product_coefficient(dims, c, k),
            b=(float(b[0]), float(b[1]), 0.0), r_poly=REACTION_U2_1MU,
            u0=smooth_initial_state(dims, noise=1e-3, rng=np.random.default_rng((seed, i))),
            tau=T / m, m=int(m), scheme=scheme, extra=dict(c=c, k=k, b=(float(b[0]), float(b[1])))))
    return out


REACTION_U_1PU2 = (0.0, 1.0, 0.0, 1.0)  # r(u) = u (1 + u^2)


def config_e4(n=60, b=-0.01, scheme="lawson2a", m=64, T=0.25):
    """The paper's three-dimensional experiment (Section 5.2, Eq. (adr3d)): a Lap u +
    b (d_1 + d_2 + d_3) u + u (1 + u^2) on (0,1)^3, Dirichlet on the faces x_mu = 0 and
    Neumann on the faces x_mu = 1, a = exp(-|x - 1/2|^2) / 10, the smooth datum
    (27/4)^3 x1 x2 x3 (1-x1)^2 (1-x2)^2 (1-x3)^2 without noise. Nodes x_j = j / n: the
    unknowns are j = 1..n (x_n = 1), the coefficient array covers j = 0..n+1."""
    h = 1.0 / n
    xs = np.arange(0, n + 2, dtype=np.float64) * h
    X3, X2, X1 = np.meshgrid(xs, xs, xs, indexing="ij")
    a = 0.1 * np.exp(-(X1 - 0.5) ** 2 - (X2 - 0.5) ** 2 - (X3 - 0.5) ** 2)
    xi = np.arange(1, n + 1, dtype=np.float64) * h
    Y3, Y2, Y1 = np.meshgrid(xi, xi, xi, indexing="ij")
    u0 = (27.0 / 4.0) ** 3 * Y1 * Y2 * Y3 * (1 - Y1) ** 2 * (1 - Y2) ** 2 * (1 - Y3) ** 2
    return Workload(name=f"e4_{n}_{scheme}_b{b}", dims=(n, n, n), a_nodes=a, b=(b, b, b),
                    r_poly=REACTION_U_1PU2, u0=np.ascontiguousarray(u0), tau=T / m, m=int(m), scheme=scheme,
                    extra=dict(bc="mixed", form="adelta"))


def config_e3(n=256, scheme="lawson2a", m=256, T=4.0):
    """The paper's two-dimensional experiment (Section 5.1, Eq. (ad2d)): periodic on
    (-3 pi, 3 pi)^2, a = diag(1/2 + sin^2 x1 sin^2 x2 / 6, 1/2 + cos^2 x1 cos^2 x2 / 6),
    b = (sin^2 x1 / 5, sin^2 x2 / 5), r(u) = u (1 - u) / 4, u0 = exp(-(x1^2 + x2^2)), on
    n x n Fourier nodes x_j = -3 pi + j 6 pi / n. Returns (workload, L, a_diag, b_field)."""
    L = 6.0 * np.pi
    x = -3.0 * np.pi + np.arange(n, dtype=np.float64) * (L / n)
    X2, X1 = np.meshgrid(x, x, indexing="ij")
    a11 = 0.5 + np.sin(X1) ** 2 * np.sin(X2) ** 2 / 6.0
    a22 = 0.5 + np.cos(X1) ** 2 * np.cos(X2) ** 2 / 6.0
    b1 = np.sin(X1) ** 2 / 5.0
    b2 = np.sin(X2) ** 2 / 5.0
    u0 = np.exp(-(X1 ** 2 + X2 ** 2))
    w = Workload(name=f"e3_{n}_{scheme}", dims=(n, n), a_nodes=None, b=(0.0, 0.0, 0.0),
                 r_poly=(0.0, 0.25, -0.25, 0.0), u0=np.ascontiguousarray(u0), tau=T / m, m=int(m),
                 scheme=scheme, extra=dict(periodic=True, L=L))
    return w, L, [a11, a22], [b1, b2]


def periodic_instance(dims, L=2.0 * np.pi, scheme="lawson2a", m=8, T=0.05, seed=5):
    """A seeded periodic instance of the form of config_e3 in 2-D or 3-D on (0, L)^d with
    n_mu Fourier nodes x_j = j L / n_mu: a_mumu = 1/2 + (1/6) prod_nu sin^2(x_nu + phase),
    b_mu = (1/5) sin^2(x_mu + phase) (random phases), r(u) = u (1 - u) / 4 and a smooth
    random datum (the lowest three modes per direction with N(0,1) amplitudes, plus 1/2).
    Returns (workload, L, a_diag, b_field)."""
    rng = np.random.default_rng(seed)
    d = len(dims)
    axes = [np.arange(n, dtype=np.float64) * (L / n) for n in dims]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]     # grids[mu] varies along x_(mu+1)
    w0 = 2.0 * np.pi / L
    a_diag, b_field = [], []
    for mu in range(d):
        ph = rng.uniform(0, 2 * np.pi, size=d)
        prod = np.ones(grids[0].shape)
        for nu in range(d):
            prod = prod * np.sin(w0 * grids[nu] + ph[nu]) ** 2
        a_diag.append(0.5 + prod / 6.0)
        b_field.append(np.sin(w0 * grids[mu] + rng.uniform(0, 2 * np.pi)) ** 2 / 5.0)
    u0 = np.full(grids[0].shape, 0.5)
    for mu in range(d):
        for kk in range(1, 4):
            if kk < dims[mu] // 2:
                c, s = rng.standard_normal(2) * 0.1
                u0 = u0 + c * np.cos(kk * w0 * grids[mu]) + s * np.sin(kk * w0 * grids[mu])
    w = Workload(name="periodic_" + "x".join(str(n) for n in dims) + f"_{scheme}", dims=tuple(dims), a_nodes=None,
                 b=(0.0, 0.0, 0.0), r_poly=(0.0, 0.25, -0.25, 0.0), u0=np.ascontiguousarray(u0), tau=T / m,
                 m=int(m), scheme=scheme, extra=dict(periodic=True, L=L))
    return w, L, a_diag, b_field


def config_e2(n=1024, scheme="lawson_euler", m=4096, T=0.1, embed=False):
    """The paper's one-dimensional nonlinear diffusion-reaction problem (Section 4, Eq.
    (adnonlinear)): u_t = (a u_x)_x + u (1 - u) on (-pi, pi), periodic, a = 1 + 10 sin^2 x,
    u0 = sin x, on n Fourier nodes x_j = -pi + j 2 pi / n. With embed=True the problem is given
    on n x 2 nodes, constant along x2 (a_22 = a_11, b = 0): the x2 direction then has only the
    mean and the Nyquist mode, whose first derivative is 0, so the solution stays the 1-D one.
    Returns (workload, L, a_diag, b_field)."""
    L = 2.0 * np.pi
    x = -np.pi + np.arange(n, dtype=np.float64) * (L / n)
    a = 1.0 + 10.0 * np.sin(x) ** 2
    u0 = np.sin(x)
    dims, a_diag, b_field = (n,), [a], [np.zeros(n)]
    if embed:
        dims = (n, 2)
        a2 = np.stack([a, a])
        a_diag, b_field, u0 = [a2, a2], [np.zeros((2, n)), np.zeros((2, n))], np.stack([u0, u0])
    w = Workload(name=f"e2_{n}_{scheme}", dims=dims, a_nodes=None, b=(0.0, 0.0, 0.0),
                 r_poly=(0.0, 1.0, -1.0, 0.0), u0=np.ascontiguousarray(u0), tau=T / m, m=int(m), scheme=scheme,
                 extra=dict(periodic=True, L=L))
    return w, L, a_diag, b_field


def config_e1(n=4096, scheme="lawson_euler", m=64, T=1.0 / 40.0, embed=False):
    """The paper's one-dimensional linear diffusion problem (Section 4, Eq. (adlinearzero)):
    u_t = a(x) u_xx on (-pi, pi), periodic, a = 1 + 10 sin^2 x, u0 = sin x, on n Fourier nodes
    x_j = -pi + j 2 pi / n (the a Lap u form, no advection, no reaction). embed=True gives it on
    n x 2 nodes, constant along x2, as config_e2 does. Returns (workload, L, a_diag, b_field)."""
    w, L, a_diag, b_field = config_e2(n=n, scheme=scheme, m=m, T=T, embed=embed)
    w.name = f"e1_{n}_{scheme}"
    w.r_poly = (0.0, 0.0, 0.0, 0.0)
    w.extra = dict(periodic=True, L=L, form="adelta")
    return w, L, a_diag, b_field

"""Every single-grid benchmark workload at its full size, through the launch path the benchmark
times (adr_integrate: the 8-step CUDA graph replayed, plus the 1-step graph for the rest),
against the FP64 oracle.

Covered: the 32^2 workloads (Lawson-Euler, ETD2RK), the paper's three-dimensional experiment
(N = 60, T = 1/4, b = -0.01, 2^8 steps; Lawson2a and stabilized Lawson2), its two-dimensional
periodic one (256^2 Fourier nodes, 2^8 steps to T = 4; Lawson2a, ETD2RK, Lawson4) and the same
problem on 1024^2 nodes, and the two 1-D experiments on n x 2 nodes. The 128^3 workload has its
own full-size test in test_gpu_parity.py. The 384^3 workloads have no oracle comparison: their
solution falls below 1e-28 within a dozen steps (b = 50 carries it out of the box), so an error
at T = 1 measures nothing.

Tolerances (relative l2):
  * FP64: 1e-11, as for the other FP64 time integrations (the spectral derivative amplifies the
    FFT's rounding by up to k_max^2 once per step, and e^{tau A} damps it again).
  * The mixed path (E4, FP32 state, tensor-core contractions): 2e-6. One step leaves a relative
    error of about 4e-8 on this grid (the FP32 state, and its slices, whose resolution is 2^-32
    of the state's max-abs). The contraction is unbiased (ten products into exact accumulators,
    a 32-bit factor), so the errors of successive steps are independent and grow as sqrt(m):
    4e-8 x 16 = 6.4e-7 at 2^8 steps. With six products, two accumulators and a 24-bit factor,
    the factor's fixed representation error made it grow linearly, to 1.9e-4 at 2^8 steps.
  * FP32 on the 1024^2 periodic problem: 1e-4, the bound derived for the 256^2 FP32 test in
    test_gpu_periodic.py (fewer steps here, and k_max^2 grows by 16 while tau shrinks by 4).
"""
import numpy as np
import pytest

from oracle import adr_oracle as O
from parity import assert_parity
import bench

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2303_15861_gb300 import adr, build_lib, workloads as W  # noqa: E402

build_lib.build()
adr.load_library()

TOL = {"fp64": 1e-11, "bf16x3": 2e-6, "fp32": 1e-4}
_REF = {}


def load(name):
    make, default_prec = bench.GRID_WORKLOADS[name]
    w = make(W)
    if isinstance(w, tuple):
        return w, default_prec
    return (w, None, None, None), default_prec


def oracle_solution(name):
    if name not in _REF:
        (w, L, a_diag, b_field), _ = load(name)
        if L is not None:
            _REF[name] = O.solve_periodic(w.dims, L, a_diag, b_field, w.r_poly, w.u0, w.tau, w.m, w.scheme,
                                          form=w.extra.get("form", "flux"))
        else:
            kw = {k: w.extra[k] for k in ("bc", "form") if k in w.extra}
            _REF[name] = O.solve(w.dims, w.a_nodes, w.b, w.r_poly, w.u0, w.tau, w.m, w.scheme, **kw)
    return _REF[name]


def gpu_solution(name, prec):
    (w, L, a_diag, b_field), _ = load(name)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        if L is not None:
            ctx = adr.Context(w.dims, w.tau, w.scheme, prec, stream=s, periodic=True, length=L,
                              form=w.extra.get("form", "flux"))
            ctx.set_coeffs_periodic(a_diag, b_field, w.r_poly)
        else:
            kw = {k: w.extra[k] for k in ("bc", "form") if k in w.extra}
            ctx = adr.Context(w.dims, w.tau, w.scheme, prec, stream=s, **kw)
            ctx.set_coeffs(w.a_nodes, w.b, w.r_poly)
        u = torch.tensor(w.u0, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
        ctx.integrate(u, 0.0, 0.0, w.m)        # T = 0: m steps of the context's tau
        ctx.synchronize()
        out = u.double().cpu().numpy()
        ctx.close()
    return out


CASES = [("c1-le", "fp64"), ("c1-etd2rk", "fp64"),
         ("e4-lawson2a", "fp64"), ("e4-lawson2a", "bf16x3"),
         ("e4-stabilized-lawson2", "fp64"), ("e4-stabilized-lawson2", "bf16x3"),
         ("e3-lawson2a", "fp64"), ("e3-etd2rk", "fp64"), ("e3-lawson4", "fp64"),
         ("e3-lawson2a-1024", "fp64"), ("e3-lawson2a-1024", "fp32"),
         ("e1-lawson-euler", "fp64"), ("e2-lawson2a", "fp64")]


def test_every_single_grid_workload_but_the_384_cube_is_covered():
    covered = {name for name, _ in CASES} | {"c2"}
    assert set(bench.GRID_WORKLOADS) - covered == {"c5-lawson4", "c5-etd2rk"}


@pytest.mark.parametrize("name,prec", CASES)
def test_bench_workload_matches_oracle(name, prec):
    got = gpu_solution(name, prec)
    ref = oracle_solution(name)
    err, err_inf, _ = assert_parity(got, ref, TOL[prec], what=f"{name} {prec}")
    print(f"{name} {prec}: rel l2 vs oracle {err:.3e}, rel max {err_inf:.3e}")


def test_the_standard_tensor_core_factors_have_four_slices():
    """The paper's 3-D experiment (tau a / h^2 = 0.36: e^{c tau A_mu} close to the identity) and
    the 256^3 Lawson4 workload (tau a / h^2 = 248) both get 32-bit factors; FP64 contexts have
    no tensor-core images."""
    (w, _, _, _), _ = load("e4-lawson2a")
    c = adr.Context(w.dims, w.tau, w.scheme, "bf16x3", bc="mixed", form="adelta")
    c.set_coeffs(w.a_nodes, w.b, w.r_poly)
    assert c.tc_factor_slices() == 4
    c.close()
    w3 = W.config3()
    c = adr.Context(w3.dims, w3.tau, "lawson4", "bf16x3")
    c.set_coeffs(w3.a_nodes, w3.b, w3.r_poly)
    assert c.tc_factor_slices() == 4
    c.close()
    c = adr.Context(w3.dims, w3.tau, "lawson4", "fp64")
    c.set_coeffs(w3.a_nodes, w3.b, w3.r_poly)
    assert c.tc_factor_slices() == 0
    c.close()

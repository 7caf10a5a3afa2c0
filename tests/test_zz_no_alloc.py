"""adr_mumode_apply_static: the mu-mode chain for callers that cannot allocate device memory.

Some callers of this library cannot call cudaMalloc: applications that reserve all of
their device memory up front in their own pool, or pipelines in which an allocation would
synchronise the device. For them the library offers one entry point that allocates
nothing and keeps its intermediates in a fixed static device array. This test checks,
through the C ABI, that two calls in a row give the same result as the context-based
entry point adr_apply_exp (the one that uses library workspace) and as the FP64 oracle's
mu-mode exponential action (Section 1), element by element within the FP64 tolerance of
the other parity tests; that a grid of exactly the static array's 1,048,576 points is
accepted; and that larger grids are refused.
"""
import numpy as np
import pytest

from oracle import adr_oracle as O
from paper_2303_15861_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2303_15861_gb300 import adr, build_lib  # noqa: E402

build_lib.build()
adr.load_library()

TOL = 1e-13   # FP64 exp-action tolerance of tests/test_gpu_parity.py (relative l2 and max norm)


def _case(dims, c, tau, seed):
    a = W.sine_product_coefficient(dims)
    b = (10.0, -7.0, 4.0)[: len(dims)]
    r = W.REACTION_U2_1MU
    ctx = adr.Context(dims, tau, "lawson4", "fp64")
    ctx.set_coeffs(a, b, r)
    # the same factors e^{c tau A_mu}, built independently on the host
    prob = O.ADRProblem(dims, a, b, r)
    factors = [torch.tensor(O.expm(c * tau * prob.factor(mu)), device="cuda")
               for mu in range(1, len(dims) + 1)]
    v_host = np.random.default_rng(seed).standard_normal(tuple(dims[::-1]))
    v = torch.tensor(v_host, device="cuda")
    oracle = O.MatrixFunctions(prob, tau).exp_action(c, v_host)
    return ctx, factors, v, oracle


def _check(y, ref):
    got = y.cpu().numpy()
    assert np.isfinite(got).all()
    assert O.rel_l2(got, ref) < TOL
    assert O.rel_inf(got, ref) < TOL


@pytest.mark.parametrize("cases", [
    [((45, 19, 23), 0.5, 2.5e-3, 1), ((70, 45), 1.0, 2e-3, 2)],
    [((128, 128, 64), 0.5, 2.5e-3, 3)],          # exactly the static array: 1,048,576 points
], ids=["small", "at_the_limit"])
def test_static_chain_matches_context_entry_point_and_oracle_twice_in_a_row(cases):
    results = []
    for dims, c, tau, seed in cases:
        for _ in range(2):                       # two calls in a row share the static array
            ctx, factors, v, oracle = _case(dims, c, tau, seed)
            y_ref = torch.empty_like(v)
            ctx.apply_exp(c, v, y_ref)
            y = torch.full_like(v, float("nan"))
            adr.adr_mumode_apply_static(factors, v, y)
            torch.cuda.synchronize()
            results.append((y, y_ref, oracle))
            ctx.close()
    for y, y_ref, oracle in results:
        _check(y, y_ref.cpu().numpy())          # the context-based entry point
        _check(y, oracle)                        # the FP64 oracle


def test_static_chain_refuses_grids_beyond_the_static_array():
    dims = (128, 128, 65)   # 1,064,960 points > 1,048,576
    factors = [torch.eye(n, dtype=torch.float64, device="cuda") for n in dims]
    v = torch.zeros(dims[::-1], dtype=torch.float64, device="cuda")
    y = torch.zeros_like(v)
    with pytest.raises(adr.AdrError) as e:
        adr.adr_mumode_apply_static(factors, v, y)
    assert e.value.status == 1

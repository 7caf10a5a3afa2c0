"""adr_mumode_apply_static: the mu-mode chain for callers that cannot allocate device memory.

Some callers of this library cannot call cudaMalloc: applications that reserve all of
their device memory up front in their own pool, or pipelines in which an allocation would
synchronise the device. For them the library offers one entry point that allocates
nothing and keeps its intermediates in a fixed static device array. This test checks,
through the C ABI, that two calls in a row give the same result as the context-based
entry point adr_apply_exp (the one that uses library workspace), within the FP64
tolerance of the other parity tests, and that grids beyond the static array are refused.
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

TOL = 1e-13   # FP64 exp-action tolerance of tests/test_gpu_parity.py


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
    v = torch.tensor(np.random.default_rng(seed).standard_normal(tuple(dims[::-1])), device="cuda")
    return ctx, factors, v


def test_static_chain_matches_context_entry_point_twice_in_a_row():
    cases = [((45, 19, 23), 0.5, 2.5e-3, 1), ((70, 45), 1.0, 2e-3, 2)]
    results = []
    for dims, c, tau, seed in cases:
        ctx, factors, v = _case(dims, c, tau, seed)
        y_ref = torch.empty_like(v)
        ctx.apply_exp(c, v, y_ref)
        y = torch.full_like(v, float("nan"))
        adr.adr_mumode_apply_static(factors, v, y)
        torch.cuda.synchronize()
        results.append((y, y_ref))
    for y, y_ref in results:
        err = O.rel_l2(y.cpu().numpy(), y_ref.cpu().numpy())
        assert err < TOL, err


def test_static_chain_refuses_grids_beyond_the_static_array():
    dims = (128, 128, 65)   # 1,064,960 points > 1,048,576
    factors = [torch.eye(n, dtype=torch.float64, device="cuda") for n in dims]
    v = torch.zeros(dims[::-1], dtype=torch.float64, device="cuda")
    y = torch.zeros_like(v)
    with pytest.raises(adr.AdrError) as e:
        adr.adr_mumode_apply_static(factors, v, y)
    assert e.value.status == 1

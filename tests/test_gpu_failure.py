"""Failure detection without a GPU fault: a device wait that nothing completes gives up after a
short limit, the host sees ADR_ERR_TIMEOUT on the next synchronize, the error word is cleared,
and the context keeps producing correct steps."""
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


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_bounded_wait_timeout_is_reported_and_the_context_recovers(prec):
    w = W.config2(n=32, m=2, scheme="lawson4")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx = adr.Context(w.dims, w.tau, w.scheme, prec, stream=s)
        ctx.set_coeffs(w.a_nodes, w.b, w.r_poly)
        dt = torch.float64 if prec == "fp64" else torch.float32
        u = torch.tensor(w.u0, dtype=dt, device="cuda")
        ctx.step(u)
        ctx.synchronize()
        adr.adr_test_bounded_wait(ctx.ctx, 1.0)          # a wait that runs out after about 1 ms
        with pytest.raises(adr.AdrError) as e:
            ctx.synchronize()
        assert e.value.status == 6                       # ADR_ERR_TIMEOUT
        ctx.synchronize()                                # the word was cleared
        u.copy_(torch.tensor(w.u0, dtype=dt))
        ctx.integrate(u, 0.0, 2 * w.tau, 2)
        ctx.synchronize()
    ref = O.solve(w.dims, w.a_nodes, w.b, w.r_poly, w.u0, w.tau, 2, w.scheme)
    assert_parity(u.double().cpu().numpy(), ref, (1e-12 if prec == "fp64" else 2e-6))

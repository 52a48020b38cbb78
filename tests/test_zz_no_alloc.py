"""The allocation-free solve, for callers that cannot allocate device memory
(applications that own all device memory through their own pool, or code
that cannot accept cudaMalloc's implicit synchronization).

It must give the same answer as pdds_solve, call after call, although every
call reuses one static scratch array per device.  This file is collected last
so that a run stopping at its first failure has already run everything else.
"""
import numpy as np
import pytest

from paper_2301_05780_gb300 import pdds, workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("w", [W.config1(), W.config2().scaled(n_paths=2000)],
                         ids=["cfg1", "cfg2"])
def test_noalloc_solve_matches_pdds_solve_twice(w):
    P = pdds.Problem(w)
    P.assemble()
    pdds.pdds_solve(P.ctx, P.G, P.b, P.u, rtol=1e-12, maxit=5000)
    ref = P.u.clone()
    for _ in range(2):          # two calls in a row share the static scratch
        u = torch.full_like(P.u, float("nan"))
        it = pdds.pdds_solve_noalloc(P.G, P.b, u, rtol=1e-12, maxit=5000)
        torch.cuda.synchronize()
        assert it > 0
        assert torch.allclose(u, ref, rtol=1e-9, atol=1e-11)


def test_noalloc_solve_rejects_too_large_systems():
    P = pdds.Problem(W.config1())
    with pytest.raises(pdds.PddsError) as e:
        pdds.pdds_solve_noalloc(P.G, P.b, P.u, n=131073)
    assert e.value.status == pdds.PDDS_EINVAL
    assert "131072" in str(e.value)

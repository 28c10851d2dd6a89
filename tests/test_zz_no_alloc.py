"""gw_grad_noalloc: the gradient for callers that cannot allocate device
memory (fixed static scratch instead of a context workspace).  Checked
against gw_grad on two calls in a row, through the C ABI.

This file sorts last so that a run stopping at the first failure has run
every other test before it."""
import numpy as np
import pytest

from paper_2404_08970_gb300 import inputs as I
from tests import gwtest_util as U

pytestmark = pytest.mark.gpu


def test_noalloc_matches_gw_grad_on_two_calls():
    import torch
    from paper_2404_08970_gb300 import _lib as L
    U.ctx()  # builds and loads the library, creates the reference context
    cases = [(1024, 768, 1, "target"), (600, 2048, 2, "exact")]
    for n, m, k, marg in cases:
        rng = np.random.default_rng(n + m)
        u, v = I.dirichlet(n, 1.0, rng), I.dirichlet(m, 1.0, rng)
        T = I.random_coupling(u, v, rng).astype(np.float32)
        dT = torch.from_numpy(T).cuda()
        du, dv = torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda()
        G_ref = torch.empty_like(dT)
        G_na = torch.full_like(dT, float("nan"))
        prob = L.problem(dim=1, nx=n, ny=m, hx=1.0 / n, hy=1.0 / m, k=k, dtype=L.GW_F32)
        mg = L.GW_MARG_TARGET if marg == "target" else L.GW_MARG_EXACT
        U.ctx().gw_grad(prob, du, dv, dT, G_ref, mg)
        b = G_ref.double().cpu().numpy()
        for _ in range(2):  # the second call reuses the scratch the first one left behind
            G_na.fill_(float("nan"))
            L.gw_grad_noalloc(prob, du, dv, dT, G_na, mg)
            torch.cuda.synchronize()
            a = G_na.double().cpu().numpy()
            assert np.all(np.isfinite(a))
            assert U.relerr(a, b) <= 1e-6
            # The same kernels on the same inputs: the results are identical.
            assert torch.equal(G_na, G_ref)


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch
    from paper_2404_08970_gb300 import _lib as L
    n = m = 16384
    prob = L.problem(dim=1, nx=n, ny=m, hx=1.0 / n, hy=1.0 / m, k=1, dtype=L.GW_F32)
    T = torch.empty(1, device="cuda")
    G = torch.empty(1, device="cuda")
    with pytest.raises(L.GWError) as e:
        # Sizes are checked before any device work; the tiny buffers are never touched.
        L.gw_grad_noalloc(prob, None, None, T, G, L.GW_MARG_EXACT)
    assert e.value.status == L.GW_ERR_INVALID


@pytest.mark.parametrize("hx", [float("inf"), float("nan"), 0.0, -1.0])
def test_noalloc_rejects_bad_spacing(hx):
    import torch
    from paper_2404_08970_gb300 import _lib as L
    prob = L.problem(dim=1, nx=8, ny=8, hx=hx, hy=0.125, k=1, dtype=L.GW_F32)
    T = torch.empty(8, 8, device="cuda")
    G = torch.empty(8, 8, device="cuda")
    with pytest.raises(L.GWError) as e:
        L.gw_grad_noalloc(prob, None, None, T, G, L.GW_MARG_EXACT)
    assert e.value.status == L.GW_ERR_INVALID

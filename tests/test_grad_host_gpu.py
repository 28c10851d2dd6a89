"""gw_grad_host (host buffers in and out, copies pipelined over two device
slots) gives exactly gw_grad's result, call after call, with page-locked
and with pageable host buffers, 1D and 2D."""
import numpy as np
import pytest

from paper_2404_08970_gb300 import inputs as I
from tests import gwtest_util as U

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pinned", [True, False])
def test_grad_host_equals_gw_grad(pinned):
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    n, m, k = 700, 1100, 2
    rng = np.random.default_rng(71)
    u, v = I.dirichlet(n, 1.0, rng), I.dirichlet(m, 1.0, rng)
    Ts = [I.random_coupling(u, v, rng).astype(np.float32) for _ in range(3)]
    prob = L.problem(dim=1, nx=n, ny=m, hx=1.0 / n, hy=1.0 / m, k=k, dtype=L.GW_F32)
    hT = [torch.from_numpy(T) for T in Ts]
    hG = [torch.full((n, m), float("nan")) for _ in Ts]
    if pinned:
        hT = [t.pin_memory() for t in hT]
        hG = [t.pin_memory() for t in hG]
    hu, hv = torch.from_numpy(u), torch.from_numpy(v)
    stream = torch.cuda.current_stream()
    # Five calls in a row (slots reused), the caller's stream synchronised once.
    order = [0, 1, 2, 0, 1]
    for i in order:
        c.gw_grad_host(prob, hu, hv, hT[i], hG[i], L.GW_MARG_TARGET, stream)
    c.gw_ctx_check(stream)
    du, dv = hu.cuda(), hv.cuda()
    for i, T in enumerate(Ts):
        dT = torch.from_numpy(T).cuda()
        dG = torch.empty_like(dT)
        c.gw_grad(prob, du, dv, dT, dG, L.GW_MARG_TARGET)
        c.gw_ctx_check()
        assert torch.equal(hG[i], dG.cpu()), i


def test_grad_host_2d_exact_marginals():
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    rng = I.rng_for(72)
    u, v = I.abs_normal_image(12, rng), I.abs_normal_image(9, rng)
    T = I.random_coupling(u, v, rng)
    prob = L.problem(dim=2, nx=12, ny=9, hx=1 / 11, hy=1 / 8, k=1, cost=L.GW_COST_SQEUCLID, dtype=L.GW_F64)
    G = np.empty_like(T)
    c.gw_grad_host(prob, None, None, T, G, L.GW_MARG_EXACT)
    c.gw_ctx_check()
    dT = torch.from_numpy(T).cuda()
    dG = torch.empty_like(dT)
    c.gw_grad(prob, None, None, dT, dG, L.GW_MARG_EXACT)
    c.gw_ctx_check()
    assert np.array_equal(G, dG.cpu().numpy())


def test_grad_host_rejects_bad_arguments():
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    T = np.zeros((4, 4), dtype=np.float32)
    prob = L.problem(dim=1, nx=4, ny=4, hx=0.25, hy=0.25, k=1, dtype=L.GW_F32)
    with pytest.raises(L.GWError) as e:
        c.gw_grad_host(prob, None, None, T, T, L.GW_MARG_EXACT)   # G overlaps T
    assert e.value.status == L.GW_ERR_INVALID
    with pytest.raises(L.GWError) as e:
        c.gw_grad_host(prob, None, None, T, np.empty_like(T), L.GW_MARG_TARGET)  # no marginals
    assert e.value.status == L.GW_ERR_INVALID

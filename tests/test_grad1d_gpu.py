"""Parity of the structured 1D gradient (CUDA, through the C ABI) with the FP64
oracle.  Tolerances: relative error max|G - G*| / max|G*| <= 1e-6 for float
arithmetic, <= 1e-12 for double."""
import numpy as np
import pytest

from paper_2404_08970_gb300 import inputs as I
from tests import gwtest_util as U

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-6, "f64": 1e-12}

# (70, 1056) and (40, 6144): rows fed by TMA (m a multiple of 32) with the last
# warps of the row partly or wholly past m.
SHAPES = [(1, 1), (1, 7), (5, 1), (3, 5), (17, 33), (64, 64), (100, 257), (200, 200), (513, 300), (1000, 1023),
          (257, 2049), (300, 4100), (70, 1056), (40, 6144)]


def _case(n, m, seed, alpha=1.0):
    rng = np.random.default_rng(seed)
    u = I.dirichlet(n, alpha, rng)
    v = I.dirichlet(m, alpha, rng)
    T = I.random_coupling(u, v, rng)
    return u, v, T


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}")
def test_grad1d_parity(shape, k, dtype):
    n, m = shape
    u, v, T = _case(n, m, 1000 * k + n + m)
    hx, hy = 1.0 / n, 1.0 / m
    Tc = T.astype(np.float32) if dtype == "f32" else T
    for marg in ("target", "exact"):
        G = U.gpu_grad_1d(Tc, u, v, k, hx, hy, dtype, marg)
        Gs = U.oracle_grad_1d(Tc.astype(np.float64), u, v, k, hx, hy, marg)
        err = U.relerr(G, Gs)
        assert err <= TOL[dtype], f"{marg} rel err {err:.3e}"


@pytest.mark.parametrize("k", [1, 2])
def test_grad1d_wide_rows(k):
    """m above 8192 uses the 1024-thread row layout."""
    n, m = 40, 9001
    u, v, T = _case(n, m, 77 + k)
    Tc = T.astype(np.float32)
    G = U.gpu_grad_1d(Tc, u, v, k, 1.0 / n, 1.0 / m, "f32", "target")
    Gs = U.oracle_grad_1d(Tc.astype(np.float64), u, v, k, 1.0 / n, 1.0 / m, "target")
    assert U.relerr(G, Gs) <= TOL["f32"]


def test_grad1d_nonuniform_spacing_and_mass():
    """Unnormalised positive T, different spacings: G is linear in T, so the
    kernel must not assume a probability coupling."""
    rng = np.random.default_rng(5)
    n, m = 150, 97
    T = I.random_positive(n, m, rng) * 3.7
    for k in (1, 2):
        G = U.gpu_grad_1d(T.astype(np.float32), None, None, k, 0.37, 2.1, "f32", "exact")
        Gs = U.oracle_grad_1d(T.astype(np.float32).astype(np.float64), None, None, k, 0.37, 2.1, "exact")
        assert U.relerr(G, Gs) <= TOL["f32"]


@pytest.mark.parametrize("marg_kind", ["uniform", "dirichlet"])
@pytest.mark.parametrize("k", [1, 2])
def test_grad1d_full_size_sampled(k, marg_kind):
    """n = m = 8192 (the benchmark workload, same launch path): sampled rows
    against the oracle, including band boundaries and both ends."""
    w = I.workload_1d_grad(8192, k, marg_kind, seed=0)
    T32 = w["T"].astype(np.float32)
    G = U.gpu_grad_1d(T32, w["u"], w["v"], k, w["hx"], w["hy"], "f32", "target")
    rows = [0, 1, 53, 54, 55, 4095, 4096, 8190, 8191]
    Gs = U.oracle_grad_rows_1d(T32.astype(np.float64), rows, w["u"], w["v"], k, w["hx"], w["hy"])
    err = U.relerr(G[rows], Gs)
    assert err <= TOL["f32"], f"sampled rel err {err:.3e}"
    # Property at full size: reflecting T reflects G (exact symmetry of the grid).
    Gr = U.gpu_grad_1d(np.ascontiguousarray(T32[::-1, ::-1]), w["u"][::-1].copy(), w["v"][::-1].copy(), k,
                       w["hx"], w["hy"], "f32", "target")
    assert U.relerr(Gr[::-1, ::-1], G) <= 2 * TOL["f32"]


def test_grad1d_invalid_arguments():
    from paper_2404_08970_gb300 import _lib as L
    import torch
    c = U.ctx()
    T = torch.ones(4, 4, device="cuda")
    G = torch.empty_like(T)
    bad = [L.problem(dim=1, nx=0, ny=4), L.problem(dim=1, nx=4, ny=4, k=0), L.problem(dim=1, nx=4, ny=4, hx=-1.0),
           L.problem(dim=3, nx=4, ny=4), L.problem(dim=1, nx=4, ny=4, dtype=7)]
    for p in bad:
        with pytest.raises(L.GWError) as e:
            c.gw_grad(p, None, None, T, G, L.GW_MARG_EXACT)
        assert e.value.status == L.GW_ERR_INVALID
    p = L.problem(dim=1, nx=4, ny=4)
    with pytest.raises(L.GWError):
        c.gw_grad(p, None, None, T, T, L.GW_MARG_EXACT)  # overlap
    with pytest.raises(L.GWError):
        c.gw_grad(p, None, None, T, G, L.GW_MARG_TARGET)  # missing marginals


def test_grad1d_generic_row_kernel():
    """The block-scan row kernel (used for k = 3 and rows above 8192) on the
    k = 1, 2 cases the warp-specialised kernel normally takes."""
    import os
    from paper_2404_08970_gb300 import _lib as L
    import torch
    os.environ["GW_FORCE_GENERIC"] = "1"
    try:
        c = L.Context(0)
    finally:
        del os.environ["GW_FORCE_GENERIC"]
    for (n, m, k) in [(100, 257, 1), (64, 1024, 2), (300, 4096, 1), (129, 8192, 2)]:
        u, v, T = _case(n, m, 31 * n + k)
        Tc = T.astype(np.float32)
        dT = torch.from_numpy(Tc).cuda()
        dG = torch.empty_like(dT)
        prob = L.problem(dim=1, nx=n, ny=m, hx=1.0 / n, hy=1.0 / m, k=k, dtype=L.GW_F32)
        c.gw_grad(prob, torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), dT, dG, L.GW_MARG_TARGET)
        c.gw_ctx_check()
        Gs = U.oracle_grad_1d(Tc.astype(np.float64), u, v, k, 1.0 / n, 1.0 / m, "target")
        assert U.relerr(dG.double().cpu().numpy(), Gs) <= TOL["f32"], (n, m, k)
    c.close()


@pytest.mark.parametrize("n,m,k", [(24, 8192, 1), (8192, 24, 2)])
def test_grad1d_peaked_late_iterate_plan(n, m, k):
    """The plan the solver actually hands to the gradient: a late mirror-descent
    iterate of the FP64 oracle at eps = 5e-3 (20 x 100), whose entries span
    many orders of magnitude (nearly empty rows and columns included), rounded
    to float32.  Target and exact marginals, 1e-6 relative."""
    from oracle import gw_oracle as O
    rng = np.random.default_rng(n + 3 * m + k)
    u, v = I.dirichlet(n, 1.0, rng), I.dirichlet(m, 1.0, rng)
    hx, hy = 1.0 / n, 1.0 / m
    DX, DY = O.grid_dist_1d(n, hx, k), O.grid_dist_1d(m, hy, k)
    T, _, _ = O.mirror_descent(DX, DY, u, v, 5e-3, 20, 100)
    Tc = T.astype(np.float32)
    pos = Tc[Tc > 0].astype(np.float64)
    assert pos.max() / pos.min() > 1e6  # peaked: many orders of magnitude
    for marg in ("target", "exact"):
        G = U.gpu_grad_1d(Tc, u, v, k, hx, hy, "f32", marg)
        Gs = U.oracle_grad_1d(Tc.astype(np.float64), u, v, k, hx, hy, marg)
        err = U.relerr(G, Gs)
        assert err <= TOL["f32"], f"{marg} rel err {err:.3e}"


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("k,ky", [(1, 2), (2, 1)])
@pytest.mark.parametrize("shape", [(1, 5), (37, 61), (300, 257), (1000, 1024), (150, 4096), (40, 8192)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
def test_grad1d_mixed_exponents(shape, k, ky, dtype):
    """k_X != k_Y (Sec. 2 takes separate exponents): D_X = h_X^k |i-j|^k,
    D_Y = h_Y^ky |p-q|^ky."""
    import torch
    from oracle import gw_oracle as O
    from paper_2404_08970_gb300 import _lib as L
    n, m = shape
    if dtype == "f64" and m > 4096:
        pytest.skip("mixed exponents in double take rows of at most 4096 columns")
    u, v, T = _case(n, m, 500 + n + m + k)
    hx, hy = 1.0 / n, 1.0 / m
    Tc = T.astype(np.float32) if dtype == "f32" else T
    c = U.ctx()
    tdt = torch.float32 if dtype == "f32" else torch.float64
    dT = torch.from_numpy(np.ascontiguousarray(Tc)).to("cuda", tdt)
    dG = torch.empty_like(dT)
    prob = L.problem(dim=1, nx=n, ny=m, hx=hx, hy=hy, k=k, ky=ky, dtype=L.GW_F32 if dtype == "f32" else L.GW_F64)
    DX, DY = O.grid_dist_1d(n, hx, k), O.grid_dist_1d(m, hy, ky)
    for marg in ("target", "exact"):
        mg = L.GW_MARG_TARGET if marg == "target" else L.GW_MARG_EXACT
        c.gw_grad(prob, torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), dT, dG, mg)
        c.gw_ctx_check()
        T64 = Tc.astype(np.float64)
        Gs = O.grad(DX, DY, T64, u, v) if marg == "target" else O.grad_exact(DX, DY, T64)
        err = U.relerr(dG.double().cpu().numpy(), Gs)
        assert err <= TOL[dtype], f"{marg} rel err {err:.3e}"


def test_grad1d_mixed_exponents_rejected_where_unsupported():
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    T = torch.zeros(4, 9000, device="cuda")
    G = torch.zeros_like(T)
    for kw in (dict(k=1, ky=3, ny=16), dict(k=1, ky=2, ny=9000), dict(k=3, ky=1, ny=16)):
        prob = L.problem(dim=1, nx=4, hx=0.25, hy=0.1, **kw)
        with pytest.raises(L.GWError) as e:
            c.gw_grad(prob, None, None, T, G, L.GW_MARG_EXACT)
        assert e.value.status == L.GW_ERR_INVALID

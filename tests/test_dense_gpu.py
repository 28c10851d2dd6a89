"""The dense comparison gradient against the FP64 oracle: the cuBLAS forms
(FP64, FP32, TF32, BF16) and the library's own tcgen05 kernels (TC TF32, TC
BF16).  FP64 and FP32 are exact up to their rounding.  The reduced-precision
forms round T, D and the intermediate product to 10 (TF32) or 7 (BF16)
mantissa bits; their measured errors on the 8192 x 8192 workload are about
4e-4 (TF32) and 1.6e-3 (BF16), and the bounds below leave a factor of about
five for other shapes."""
import numpy as np
import pytest

from paper_2404_08970_gb300 import inputs as I
from tests import gwtest_util as U

pytestmark = pytest.mark.gpu

BOUND = {"fp64": 1e-12, "fp32": 1e-5, "tf32": 2e-3, "bf16": 1e-2, "tc_tf32": 2e-3, "tc_bf16": 1e-2}


def gpu_dense(T, u, v, k, hx, hy, prec, marginals="target"):
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    tdt = torch.float64 if prec == "fp64" else torch.float32
    dT = torch.from_numpy(np.ascontiguousarray(T)).to("cuda", tdt)
    dG = torch.empty_like(dT)
    n, m = T.shape
    prob = L.problem(dim=1, nx=n, ny=m, hx=hx, hy=hy, k=k, dtype=L.GW_F64 if prec == "fp64" else L.GW_F32)
    P = {"fp32": L.GW_DENSE_FP32, "tf32": L.GW_DENSE_TF32, "bf16": L.GW_DENSE_BF16, "fp64": L.GW_DENSE_FP64,
         "tc_tf32": L.GW_DENSE_TC_TF32, "tc_bf16": L.GW_DENSE_TC_BF16}[prec]
    mg = L.GW_MARG_TARGET if marginals == "target" else L.GW_MARG_EXACT
    c.gw_grad_dense(prob, torch.from_numpy(u).cuda() if u is not None else None,
                    torch.from_numpy(v).cuda() if v is not None else None, dT, dG, mg, P)
    c.gw_ctx_check()
    return dG.double().cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16", "tc_tf32", "tc_bf16"])
@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("shape", [(64, 48), (300, 257), (1024, 1024), (257, 1001), (5, 3)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
def test_dense_parity(shape, k, prec):
    n, m = shape
    rng = np.random.default_rng(n + m + k)
    u, v = I.dirichlet(n, 1.0, rng), I.dirichlet(m, 1.0, rng)
    T = I.random_coupling(u, v, rng)
    Tc = T if prec == "fp64" else T.astype(np.float32)
    for marg in ("target", "exact"):
        G = gpu_dense(Tc, u, v, k, 1.0 / n, 1.0 / m, prec, marg)
        Gs = U.oracle_grad_1d(Tc.astype(np.float64), u, v, k, 1.0 / n, 1.0 / m, marg)
        err = U.relerr(G, Gs)
        assert err <= BOUND[prec], f"{prec} {marg} rel err {err:.3e}"


def test_dense_matches_structured_fp64():
    """FP64: the dense and the structured routes agree to rounding (the
    paper's fast = original check)."""
    n = m = 500
    rng = np.random.default_rng(3)
    u, v = I.dirichlet(n, 1.0, rng), I.dirichlet(m, 1.0, rng)
    T = I.random_coupling(u, v, rng)
    Gd = gpu_dense(T, u, v, 1, 1.0 / n, 1.0 / m, "fp64")
    Gf = U.gpu_grad_1d(T, u, v, 1, 1.0 / n, 1.0 / m, "f64", "target")
    assert U.relerr(Gf, Gd) < 1e-12


@pytest.mark.parametrize("prec", ["tc_tf32", "tc_bf16"])
def test_dense_tc_many_tiles_sampled_rows(prec):
    """4096 x 3000: both products span more 128 x 256 tiles than there are
    SMs (each persistent CTA drains one accumulator while filling the other),
    with ragged last tiles; sampled rows against the oracle."""
    n, m = 4096, 3000
    rng = np.random.default_rng(17)
    u, v = I.dirichlet(n, 1.0, rng), I.dirichlet(m, 1.0, rng)
    T = I.random_coupling(u, v, rng).astype(np.float32)
    G = gpu_dense(T, u, v, 1, 1.0 / n, 1.0 / m, prec)
    rows = [0, 1, 127, 128, 2047, 4000, 4095]
    Gs = U.oracle_grad_rows_1d(T.astype(np.float64), rows, u, v, 1, 1.0 / n, 1.0 / m)
    assert U.relerr(G[rows], Gs) <= BOUND[prec]
    assert np.all(np.isfinite(G))


@pytest.mark.parametrize("prec", ["tc_tf32", "tc_bf16"])
def test_dense_tc_2d(prec):
    """2D grids (dense distance matrices over the grid points)."""
    import torch
    from paper_2404_08970_gb300 import _lib as L
    from oracle import gw_oracle as O
    c = U.ctx()
    rng = I.rng_for(9)
    sx, sy = 12, 17
    u, v = I.abs_normal_image(sx, rng), I.abs_normal_image(sy, rng)
    T = I.random_coupling(u, v, rng).astype(np.float32)
    dT = torch.from_numpy(T).cuda()
    dG = torch.empty_like(dT)
    prob = L.problem(dim=2, nx=sx, ny=sy, hx=1 / (sx - 1), hy=1 / (sy - 1), k=1, cost=L.GW_COST_SQEUCLID,
                     dtype=L.GW_F32)
    P = L.GW_DENSE_TC_TF32 if prec == "tc_tf32" else L.GW_DENSE_TC_BF16
    c.gw_grad_dense(prob, torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), dT, dG, L.GW_MARG_TARGET, P)
    c.gw_ctx_check()
    DX = O.grid_dist_2d(sx, 1 / (sx - 1), "sqeuclid")
    DY = O.grid_dist_2d(sy, 1 / (sy - 1), "sqeuclid")
    Gs = O.grad(DX, DY, T.astype(np.float64), u, v)
    assert U.relerr(dG.double().cpu().numpy(), Gs) <= BOUND[prec]


@pytest.mark.parametrize("prec", ["fp64", "tc_bf16"])
def test_dense_mixed_exponents(prec):
    """Dense path with k_X = 1, k_Y = 2."""
    import torch
    from oracle import gw_oracle as O
    from paper_2404_08970_gb300 import _lib as L
    n, m = 96, 130
    rng = np.random.default_rng(55)
    u, v = I.dirichlet(n, 1.0, rng), I.dirichlet(m, 1.0, rng)
    T = I.random_coupling(u, v, rng)
    Tc = T if prec == "fp64" else T.astype(np.float32)
    c = U.ctx()
    dT = torch.from_numpy(np.ascontiguousarray(Tc)).cuda()
    dG = torch.empty_like(dT)
    prob = L.problem(dim=1, nx=n, ny=m, hx=1.0 / n, hy=1.0 / m, k=1, ky=2,
                     dtype=L.GW_F64 if prec == "fp64" else L.GW_F32)
    P = L.GW_DENSE_FP64 if prec == "fp64" else L.GW_DENSE_TC_BF16
    c.gw_grad_dense(prob, torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), dT, dG, L.GW_MARG_TARGET, P)
    c.gw_ctx_check()
    Gs = O.grad(O.grid_dist_1d(n, 1.0 / n, 1), O.grid_dist_1d(m, 1.0 / m, 2), Tc.astype(np.float64), u, v)
    assert U.relerr(dG.double().cpu().numpy(), Gs) <= BOUND[prec]

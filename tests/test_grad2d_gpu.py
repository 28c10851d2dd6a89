"""Parity of the 2D separable structured gradient (CUDA, through the C ABI)
with the FP64 oracle's dense definition G = (D_X o D_X) r 1^T + 1 ((D_Y o D_Y) c)^T
- 2 D_X T D_Y on side x side grids (Sec. 3.1), for the Manhattan (k = 1) and
squared Euclidean costs.

Tolerances (max |G - G*| / max |G*|): 1e-6 in float, 1e-12 in double."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2404_08970_gb300 import inputs as I
from tests import gwtest_util as U

pytestmark = pytest.mark.gpu

COSTS = {"manhattan": 0, "sqeuclid": 1}


def make(sx, sy, seed=0):
    rng = I.rng_for(seed)
    u = I.abs_normal_image(sx, rng)
    v = I.abs_normal_image(sy, rng)
    T = I.random_coupling(u, v, rng)
    return u, v, T


def gpu_grad_2d(T, u, v, sx, sy, cost, hx, hy, dtype, marginals, k=1):
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    tdt = torch.float32 if dtype == "f32" else torch.float64
    dT = torch.from_numpy(np.ascontiguousarray(T)).to("cuda", tdt)
    dG = torch.empty_like(dT)
    du = None if u is None else torch.from_numpy(np.asarray(u, dtype=np.float64)).cuda()
    dv = None if v is None else torch.from_numpy(np.asarray(v, dtype=np.float64)).cuda()
    prob = L.problem(dim=2, nx=sx, ny=sy, hx=hx, hy=hy, k=k, cost=COSTS[cost],
                     dtype=L.GW_F32 if dtype == "f32" else L.GW_F64)
    mg = L.GW_MARG_TARGET if marginals == "target" else L.GW_MARG_EXACT
    c.gw_grad(prob, du, dv, dT, dG, mg)
    c.gw_ctx_check()
    return dG.double().cpu().numpy()


def oracle_grad_2d(T64, u, v, sx, sy, cost, hx, hy, marginals, k=1):
    DX, DY = O.grid_dist_2d(sx, hx, cost, k), O.grid_dist_2d(sy, hy, cost, k)
    if marginals == "target":
        return O.grad(DX, DY, T64, u, v)
    return O.grad_exact(DX, DY, T64)


SHAPES = [(1, 1), (1, 3), (2, 3), (5, 7), (8, 12), (16, 24), (31, 33), (33, 40), (40, 64)]


@pytest.mark.parametrize("sx,sy", SHAPES)
@pytest.mark.parametrize("cost", ["manhattan", "sqeuclid"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_grad2d_matches_oracle(sx, sy, cost, dtype):
    u, v, T = make(sx, sy, seed=sx * 100 + sy)
    hx, hy = 1.0 / max(sx - 1, 1), 1.0 / max(sy - 1, 1)
    Td = T.astype(np.float32) if dtype == "f32" else T
    G = gpu_grad_2d(Td, u, v, sx, sy, cost, hx, hy, dtype, "target")
    Gs = oracle_grad_2d(Td.astype(np.float64), u, v, sx, sy, cost, hx, hy, "target")
    tol = 1e-6 if dtype == "f32" else 1e-12
    assert U.relerr(G, Gs) < tol, U.relerr(G, Gs)


@pytest.mark.parametrize("sx,sy", [(3, 4), (12, 9), (33, 35)])
@pytest.mark.parametrize("cost", ["manhattan", "sqeuclid"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_grad2d_exact_marginals(sx, sy, cost, dtype):
    """Constant term from T's own marginals, on a T that is not a coupling of
    (u, v): a plain positive array."""
    rng = I.rng_for(7)
    T = rng.uniform(0.5, 1.5, size=(sx * sx, sy * sy))
    T /= T.sum()
    Td = T.astype(np.float32) if dtype == "f32" else T
    G = gpu_grad_2d(Td, None, None, sx, sy, cost, 0.3, 0.2, dtype, "exact")
    Gs = oracle_grad_2d(Td.astype(np.float64), None, None, sx, sy, cost, 0.3, 0.2, "exact")
    tol = 1e-6 if dtype == "f32" else 1e-12
    assert U.relerr(G, Gs) < tol, U.relerr(G, Gs)


@pytest.mark.parametrize("cost", ["sqeuclid", "manhattan"])
def test_grad2d_full_size_sampled(cost):
    """64 x 64 against 96 x 96 grids (n = 4096, m = 9216, |N(0,1)| image
    marginals, unit square): 24 sampled rows against the oracle's row
    formula, all columns."""
    sx, sy = 64, 96
    u, v, T = make(sx, sy, seed=3)
    hx, hy = 1.0 / (sx - 1), 1.0 / (sy - 1)
    T32 = T.astype(np.float32)
    G = gpu_grad_2d(T32, u, v, sx, sy, cost, hx, hy, "f32", "target")
    rng = np.random.default_rng(11)
    rows = np.unique(np.concatenate([[0, sx * sx - 1, sx - 1, sx * (sx - 1)], rng.integers(0, sx * sx, 20)]))
    DX = O.grid_dist_2d(sx, hx, cost)
    DY = O.grid_dist_2d(sy, hy, cost)
    cx = (DX * DX) @ u
    cy = (DY * DY) @ v
    Gs = O.grad_rows(DX[rows], DY, T32.astype(np.float64), cx[rows], cy)
    err = float(np.max(np.abs(G[rows] - Gs)) / np.max(np.abs(Gs)))
    assert err < 1e-6, err


def test_grad2d_rejects_unsupported():
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    T = torch.zeros(16, 16, device="cuda")
    G = torch.zeros_like(T)
    u = torch.full((16,), 1 / 16, dtype=torch.float64, device="cuda")
    for kw in (dict(k=4, cost=0), dict(k=1, cost=5), dict(k=1, cost=1, nx=300), dict(k=2, cost=0, nx=129)):
        args = dict(dim=2, nx=4, ny=4, hx=0.1, hy=0.1)
        args.update(kw)
        prob = L.problem(**args)
        with pytest.raises(L.GWError) as e:
            c.gw_grad(prob, u, u, T, G, L.GW_MARG_TARGET)
        assert e.value.status == L.GW_ERR_INVALID


@pytest.mark.parametrize("cost", ["sqeuclid", "manhattan"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5), ("tf32", 2e-2), ("bf16", 1e-1)])
def test_grad2d_dense_matches_oracle(cost, precision, tol):
    """The dense comparison path on 2D grids (materialised distance matrices,
    two library matrix products) against the same oracle."""
    import torch
    from paper_2404_08970_gb300 import _lib as L
    sx, sy = 12, 16
    u, v, T = make(sx, sy, seed=2)
    hx, hy = 1.0 / (sx - 1), 1.0 / (sy - 1)
    f64 = precision == "fp64"
    Td = T if f64 else T.astype(np.float32)
    c = U.ctx()
    dT = torch.from_numpy(np.ascontiguousarray(Td)).cuda()
    dG = torch.empty_like(dT)
    prob = L.problem(dim=2, nx=sx, ny=sy, hx=hx, hy=hy, k=1, cost=COSTS[cost], dtype=L.GW_F64 if f64 else L.GW_F32)
    prec = {"fp64": L.GW_DENSE_FP64, "fp32": L.GW_DENSE_FP32, "tf32": L.GW_DENSE_TF32, "bf16": L.GW_DENSE_BF16}
    c.gw_grad_dense(prob, torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), dT, dG, L.GW_MARG_TARGET,
                    prec[precision])
    c.gw_ctx_check()
    Gs = oracle_grad_2d(Td.astype(np.float64), u, v, sx, sy, cost, hx, hy, "target")
    assert U.relerr(dG.double().cpu().numpy(), Gs) < tol


# ---------------------------------------------------------------------------
# Manhattan distance to the power k >= 2 (Sec. 3.1, eq. "2D kronecker"): the
# two-pass image-transform path.
# ---------------------------------------------------------------------------

POWK_SHAPES = [(1, 1), (1, 4), (2, 3), (5, 4), (8, 10), (16, 12), (24, 32), (13, 7)]


@pytest.mark.parametrize("sx,sy", POWK_SHAPES)
@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_grad2d_powk_matches_oracle(sx, sy, k, dtype):
    u, v, T = make(sx, sy, seed=sx * 100 + sy + 7 * k)
    hx, hy = 1.0 / max(sx - 1, 1), 1.0 / max(sy - 1, 1)
    Td = T.astype(np.float32) if dtype == "f32" else T
    tol = 1e-6 if dtype == "f32" else 1e-12
    for marg in ("target", "exact"):
        G = gpu_grad_2d(Td, u, v, sx, sy, "manhattan", hx, hy, dtype, marg, k=k)
        Gs = oracle_grad_2d(Td.astype(np.float64), u, v, sx, sy, "manhattan", hx, hy, marg, k=k)
        assert U.relerr(G, Gs) < tol, (marg, U.relerr(G, Gs))


@pytest.mark.parametrize("k", [2, 3])
def test_grad2d_powk_full_size_sampled(k):
    """64 x 64 against 96 x 96 grids, Manhattan^k: 24 sampled rows against the
    oracle's row formula, all columns."""
    sx, sy = 64, 96
    u, v, T = make(sx, sy, seed=5 + k)
    hx, hy = 1.0 / (sx - 1), 1.0 / (sy - 1)
    T32 = T.astype(np.float32)
    G = gpu_grad_2d(T32, u, v, sx, sy, "manhattan", hx, hy, "f32", "target", k=k)
    assert np.all(np.isfinite(G))
    rng = np.random.default_rng(12)
    rows = np.unique(np.concatenate([[0, sx * sx - 1, sx - 1, sx * (sx - 1)], rng.integers(0, sx * sx, 20)]))
    DX = O.grid_dist_2d(sx, hx, "manhattan", k)
    DY = O.grid_dist_2d(sy, hy, "manhattan", k)
    cx = (DX * DX) @ u
    cy = (DY * DY) @ v
    Gs = O.grad_rows(DX[rows], DY, T32.astype(np.float64), cx[rows], cy)
    err = float(np.max(np.abs(G[rows] - Gs)) / np.max(np.abs(Gs)))
    assert err < 1e-6, err


@pytest.mark.parametrize("k", [2, 3])
def test_grad2d_powk_dense_path(k):
    """The dense comparison path with Manhattan^k distance matrices."""
    import torch
    from paper_2404_08970_gb300 import _lib as L
    sx, sy = 9, 11
    u, v, T = make(sx, sy, seed=30 + k)
    hx, hy = 1.0 / (sx - 1), 1.0 / (sy - 1)
    c = U.ctx()
    dT = torch.from_numpy(T).cuda()
    dG = torch.empty_like(dT)
    prob = L.problem(dim=2, nx=sx, ny=sy, hx=hx, hy=hy, k=k, cost=0, dtype=L.GW_F64)
    c.gw_grad_dense(prob, torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), dT, dG, L.GW_MARG_TARGET,
                    L.GW_DENSE_FP64)
    c.gw_ctx_check()
    Gs = oracle_grad_2d(T, u, v, sx, sy, "manhattan", hx, hy, "target", k=k)
    assert U.relerr(dG.cpu().numpy(), Gs) < 1e-12

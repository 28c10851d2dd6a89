"""Parity of the 3D grid paths (CUDA, through the C ABI) with the FP64 oracle
on side^3 grids with the Manhattan (k = 1) and squared Euclidean costs: the
structured gradient against the dense definition G = (D_X o D_X) r 1^T +
1 ((D_Y o D_Y) c)^T - 2 D_X T D_Y (Sec. 2.1 with the 3D distance matrices of
the Sec. 3.1 construction), the mirror-descent solve, the dense comparison
path, and the argument checks.

Tolerances (max |G - G*| / max |G*|): 1e-6 in float, 1e-12 in double; solves
as in 2D (double 1e-9 on the plan, float 1e-5 on the value)."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2404_08970_gb300 import inputs as I
from tests import gwtest_util as U

pytestmark = pytest.mark.gpu

COSTS = {"manhattan": 0, "sqeuclid": 1}


def make(sx, sy, seed=0):
    rng = I.rng_for(seed)
    u = I.abs_normal_volume(sx, rng)
    v = I.abs_normal_volume(sy, rng)
    T = I.random_coupling(u, v, rng)
    return u, v, T


def _prob(L, sx, sy, cost, hx, hy, dtype, k=1, **kw):
    return L.problem(dim=3, nx=sx, ny=sy, hx=hx, hy=hy, k=k, cost=COSTS[cost],
                     dtype=L.GW_F32 if dtype == "f32" else L.GW_F64, **kw)


def gpu_grad_3d(T, u, v, sx, sy, cost, hx, hy, dtype, marginals, dense=None):
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    tdt = torch.float32 if dtype == "f32" else torch.float64
    dT = torch.from_numpy(np.ascontiguousarray(T)).to("cuda", tdt)
    dG = torch.empty_like(dT)
    du = None if u is None else torch.from_numpy(np.asarray(u, dtype=np.float64)).cuda()
    dv = None if v is None else torch.from_numpy(np.asarray(v, dtype=np.float64)).cuda()
    prob = _prob(L, sx, sy, cost, hx, hy, dtype)
    mg = L.GW_MARG_TARGET if marginals == "target" else L.GW_MARG_EXACT
    if dense is None:
        c.gw_grad(prob, du, dv, dT, dG, mg)
    else:
        c.gw_grad_dense(prob, du, dv, dT, dG, mg, precision=dense)
    c.gw_ctx_check()
    return dG.double().cpu().numpy()


def oracle_grad_3d(T64, u, v, sx, sy, cost, hx, hy, marginals):
    DX, DY = O.grid_dist_3d(sx, hx, cost), O.grid_dist_3d(sy, hy, cost)
    if marginals == "target":
        return O.grad(DX, DY, T64, u, v)
    return O.grad_exact(DX, DY, T64)


# Sides up to 13 in full (m = 2197); the row kernel's variants by the number
# of (y1, y2) pairs per lane: 1 (sy <= 5), 2 (<= 8), 4 (<= 11), 8 (<= 16).
SHAPES = [(1, 1), (1, 2), (2, 3), (3, 4), (4, 4), (5, 7), (6, 5), (8, 6), (9, 11), (11, 13)]


@pytest.mark.parametrize("sx,sy", SHAPES)
@pytest.mark.parametrize("cost", ["manhattan", "sqeuclid"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_grad3d_matches_oracle(sx, sy, cost, dtype):
    u, v, T = make(sx, sy, seed=sx * 100 + sy)
    hx, hy = 1.0 / max(sx - 1, 1), 1.0 / max(sy - 1, 1)
    Td = T.astype(np.float32) if dtype == "f32" else T
    G = gpu_grad_3d(Td, u, v, sx, sy, cost, hx, hy, dtype, "target")
    Gs = oracle_grad_3d(Td.astype(np.float64), u, v, sx, sy, cost, hx, hy, "target")
    tol = 1e-6 if dtype == "f32" else 1e-12
    assert U.relerr(G, Gs) < tol, U.relerr(G, Gs)


@pytest.mark.parametrize("sx,sy", [(3, 4), (7, 5), (10, 9)])
@pytest.mark.parametrize("cost", ["manhattan", "sqeuclid"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_grad3d_exact_marginals(sx, sy, cost, dtype):
    """Constant term from T's own marginals, on a plain positive T that is not
    a coupling of (u, v)."""
    rng = I.rng_for(11)
    T = rng.uniform(0.5, 1.5, size=(sx ** 3, sy ** 3))
    T /= T.sum()
    Td = T.astype(np.float32) if dtype == "f32" else T
    G = gpu_grad_3d(Td, None, None, sx, sy, cost, 0.3, 0.2, dtype, "exact")
    Gs = oracle_grad_3d(Td.astype(np.float64), None, None, sx, sy, cost, 0.3, 0.2, "exact")
    tol = 1e-6 if dtype == "f32" else 1e-12
    assert U.relerr(G, Gs) < tol, U.relerr(G, Gs)


def oracle_grad_cols_3d(T64, cols, u, v, sx, sy, cost, hx, hy):
    """Columns `cols` of the oracle gradient with target marginals, through the
    transpose identity G(T)[:, P] = G'(T^T)[P, :] (X and Y swapped), so that
    only D_X and the rows D_Y[P, :] are formed."""
    DX = O.grid_dist_3d(sx, hx, cost)
    DY_rows = O.grid_dist_3d_rows(sy, hy, cost, cols)
    cy_rows = (DY_rows * DY_rows) @ v
    cx = (DX * DX) @ u
    return O.grad_rows(DY_rows, DX, np.ascontiguousarray(T64.T), cy_rows, cx).T


@pytest.mark.parametrize("sx,sy", [(6, 17), (5, 23), (12, 20)])
@pytest.mark.parametrize("cost", ["manhattan", "sqeuclid"])
def test_grad3d_wide_rows_sampled(sx, sy, cost):
    """Rows of 4913 to 12167 columns (the 16- and 32-pair row-kernel variants),
    float, on 40 sampled columns including the first and last."""
    u, v, T = make(sx, sy, seed=sx + 7 * sy)
    hx, hy = 1.0 / (sx - 1), 1.0 / (sy - 1)
    Td = T.astype(np.float32)
    G = gpu_grad_3d(Td, u, v, sx, sy, cost, hx, hy, "f32", "target")
    m = sy ** 3
    cols = np.unique(np.concatenate([[0, m - 1, sy * sy - 1, sy * sy], I.rng_for(3).integers(0, m, 36)]))
    Gs = oracle_grad_cols_3d(Td.astype(np.float64), cols, u, v, sx, sy, cost, hx, hy)
    assert U.relerr(G[:, cols], Gs) < 1e-6, U.relerr(G[:, cols], Gs)


@pytest.mark.parametrize("cost", ["manhattan", "sqeuclid"])
def test_grad3d_full_workload_sampled(cost):
    """The 3D benchmark workload, 16^3 vs 21^3 (n = 4096, m = 9261), float,
    on 24 sampled columns."""
    w = I.workload_3d(16, 21, cost)
    rng = I.rng_for(1)
    T = I.random_coupling(w["u"], w["v"], rng).astype(np.float32)
    G = gpu_grad_3d(T, w["u"], w["v"], 16, 21, cost, w["hx"], w["hy"], "f32", "target")
    cols = np.unique(np.concatenate([[0, 9260, 440, 441], rng.integers(0, 9261, 20)]))
    Gs = oracle_grad_cols_3d(T.astype(np.float64), cols, w["u"], w["v"], 16, 21, cost, w["hx"], w["hy"])
    assert U.relerr(G[:, cols], Gs) < 1e-6, U.relerr(G[:, cols], Gs)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
@pytest.mark.parametrize("cost", ["manhattan", "sqeuclid"])
def test_grad3d_dense_path(prec, tol, cost):
    """The dense comparison route with explicit 3D distance matrices."""
    from paper_2404_08970_gb300 import _lib as L
    sx, sy = 5, 6
    u, v, T = make(sx, sy, seed=9)
    hx, hy = 0.25, 0.2
    dtype = "f64" if prec == "fp64" else "f32"
    Td = T if dtype == "f64" else T.astype(np.float32)
    pr = L.GW_DENSE_FP64 if prec == "fp64" else L.GW_DENSE_FP32
    G = gpu_grad_3d(Td, u, v, sx, sy, cost, hx, hy, dtype, "target", dense=pr)
    Gs = oracle_grad_3d(Td.astype(np.float64), u, v, sx, sy, cost, hx, hy, "target")
    assert U.relerr(G, Gs) < tol, U.relerr(G, Gs)


def gpu_solve_3d(w, dtype):
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    n, m = w["nx"] ** 3, w["ny"] ** 3
    tdt = torch.float32 if dtype == "f32" else torch.float64
    T = torch.empty(n, m, dtype=tdt, device="cuda")
    f = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty(m, dtype=torch.float64, device="cuda")
    stats = torch.zeros(8, dtype=torch.float64, device="cuda")
    du = torch.from_numpy(w["u"]).cuda()
    dv = torch.from_numpy(w["v"]).cuda()
    prob = _prob(L, w["nx"], w["ny"], w["cost"], w["hx"], w["hy"], dtype, eps=w["eps"], n_outer=w["n_outer"],
                 n_inner=w["n_inner"])
    c.gw_solve(prob, du, dv, T, f, g, stats)
    c.gw_ctx_check()
    return T.double().cpu().numpy(), stats.cpu().numpy()


def oracle_solve_3d(w):
    DX = O.grid_dist_3d(w["nx"], w["hx"], w["cost"])
    DY = O.grid_dist_3d(w["ny"], w["hy"], w["cost"])
    T, f, g = O.mirror_descent(DX, DY, w["u"], w["v"], w["eps"], w["n_outer"], w["n_inner"])
    return T, dict(E=O.value(DX, DY, T), H=w["eps"] * O.entropy(T))


def small_3d(sx, sy, cost, eps, n_outer, n_inner, seed):
    rng = I.rng_for(seed)
    return dict(nx=sx, ny=sy, hx=1.0 / (sx - 1), hy=1.0 / (sy - 1), cost=cost, eps=eps, n_outer=n_outer,
                n_inner=n_inner, u=I.abs_normal_volume(sx, rng), v=I.abs_normal_volume(sy, rng))


@pytest.mark.parametrize("cost", ["sqeuclid", "manhattan"])
@pytest.mark.parametrize("shape", [(3, 4), (5, 4), (6, 7)])
def test_solve3d_fp64(shape, cost):
    w = small_3d(*shape, cost, eps=5e-2, n_outer=6, n_inner=60, seed=shape[0] * 10 + shape[1])
    T, st = gpu_solve_3d(w, "f64")
    Ts, ss = oracle_solve_3d(w)
    assert U.relerr(T, Ts) < 1e-9, U.relerr(T, Ts)
    assert abs(st[1] - ss["E"]) <= 1e-10 * abs(ss["E"])
    assert abs(st[3] - ss["H"]) <= 1e-9 * abs(ss["H"])
    assert st[5] < 1e-12


@pytest.mark.parametrize("cost", ["sqeuclid", "manhattan"])
def test_solve3d_fp32_volume_workload(cost):
    """|N(0,1)| voxel marginals on the unit cube, eps = 5e-3, 20 x 100 (the 3D
    workload's schedule) on 6^3 against 7^3 grids."""
    w = small_3d(6, 7, cost, eps=5e-3, n_outer=20, n_inner=100, seed=8)
    T, st = gpu_solve_3d(w, "f32")
    Ts, ss = oracle_solve_3d(w)
    assert abs(st[1] - ss["E"]) <= 1e-5 * abs(ss["E"]), (st[1], ss["E"])
    assert st[5] < 1e-5


@pytest.mark.parametrize("kw", [dict(k=2, cost="manhattan"), dict(k=1, cost="manhattan", ky=2),
                                dict(k=1, cost="sqeuclid", sx=33), dict(k=1, cost="sqeuclid", sy=40)])
def test_grid3d_rejects_unsupported(kw):
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    sx, sy = kw.pop("sx", 4), kw.pop("sy", 4)
    k, cost = kw.pop("k"), kw.pop("cost")
    prob = _prob(L, sx, sy, cost, 0.1, 0.1, "f32", k=k, **kw)
    T = torch.zeros(sx ** 3, sy ** 3, device="cuda")
    G = torch.empty_like(T)
    with pytest.raises(L.GWError) as e:
        c.gw_grad(prob, None, None, T, G, L.GW_MARG_EXACT)
    assert e.value.status == L.GW_ERR_INVALID

"""Batched solves (gw_solve_batch): each problem's result agrees with the
single-problem solve on the same inputs (the batch uses longer row bands, so
partial sums are grouped differently: double agrees to 1e-11, float to the
1e-5 value tolerance of the solve parity tests), and the double-precision problems
match the FP64 oracle."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2404_08970_gb300 import inputs as I
from tests import gwtest_util as U

pytestmark = pytest.mark.gpu


def _prob(L, w, dtype):
    return L.problem(dim=w.get("dim", 1), nx=w["nx"], ny=w["ny"], hx=w["hx"], hy=w["hy"], k=w["k"],
                     cost=w.get("cost", 0), eps=w["eps"], n_outer=w["n_outer"], n_inner=w["n_inner"],
                     theta=w.get("theta", 1.0), feat_dim=0 if w.get("phi") is None else w["phi"].shape[1],
                     dtype=L.GW_F32 if dtype == "f32" else L.GW_F64, tau=w.get("tau", 0.0),
                     warm_start=w.get("warm", 0))


def _points(w):
    return (w["nx"] ** 2, w["ny"] ** 2) if w.get("dim", 1) == 2 else (w["nx"], w["ny"])


def _mixed():
    rng = np.random.default_rng(5)
    ws = []
    for (n, m, k) in [(37, 53, 1), (200, 180, 2), (64, 700, 1), (1500, 90, 2), (8, 8, 1), (513, 1025, 1),
                      (1, 40, 1), (300, 300, 2)]:
        ws.append(dict(nx=n, ny=m, hx=1.0 / n, hy=1.0 / m, k=k, eps=5e-2, n_outer=3, n_inner=30,
                       u=I.dirichlet(n, 1.0, rng), v=I.dirichlet(m, 1.0, rng)))
    r2 = I.rng_for(3)
    ws.append(dict(dim=2, cost="sqeuclid", nx=6, ny=9, hx=0.2, hy=0.125, k=1, eps=5e-2, n_outer=3, n_inner=30,
                   u=I.abs_normal_image(6, r2), v=I.abs_normal_image(9, r2)))
    ws.append(dict(nx=90, ny=70, hx=1 / 90, hy=1 / 70, k=1, eps=5e-2, n_outer=3, n_inner=30, tau=0.1, warm=1,
                   u=I.dirichlet(90, 1.0, rng), v=I.dirichlet(70, 1.0, rng)))
    ws.append(dict(nx=50, ny=60, hx=0.02, hy=1 / 60, k=1, eps=5e-2, n_outer=3, n_inner=30, theta=0.5,
                   u=I.dirichlet(50, 1.0, rng), v=I.dirichlet(60, 1.0, rng),
                   phi=I.features(50, 16, rng) * 0.1, psi=I.features(60, 16, rng) * 0.1))
    return ws


def _dev(ws, dtype):
    import torch
    tdt = torch.float32 if dtype == "f32" else torch.float64
    u = [torch.from_numpy(w["u"]).cuda() for w in ws]
    v = [torch.from_numpy(w["v"]).cuda() for w in ws]
    T = [torch.empty(*_points(w), dtype=tdt, device="cuda") for w in ws]
    st = [torch.zeros(8, dtype=torch.float64, device="cuda") for w in ws]
    phi = [None if w.get("phi") is None else torch.from_numpy(w["phi"]).cuda() for w in ws]
    psi = [None if w.get("psi") is None else torch.from_numpy(w["psi"]).cuda() for w in ws]
    return u, v, T, st, phi, psi


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_batch_equals_single_solves(dtype):
    import torch
    from paper_2404_08970_gb300 import _lib as L
    ws = _mixed()
    for w in ws:
        if w.get("cost") == "sqeuclid":
            w["cost"] = L.GW_COST_SQEUCLID
    c = U.ctx()
    probs = [_prob(L, w, dtype) for w in ws]
    u, v, T, st, phi, psi = _dev(ws, dtype)
    c.gw_solve_batch(probs, u, v, T, st, phi, psi)
    c.gw_ctx_check()
    for i, w in enumerate(ws):
        T1 = torch.empty_like(T[i])
        s1 = torch.zeros(8, dtype=torch.float64, device="cuda")
        c.gw_solve(probs[i], u[i], v[i], T1, None, None, s1, phi[i], psi[i])
        c.gw_ctx_check()
        a, b = T[i].double().cpu().numpy(), T1.double().cpu().numpy()
        E, E1 = float(st[i][0]), float(s1[0])
        if dtype == "f64":
            assert U.relerr(a, b) < 1e-11, i
            assert abs(E - E1) <= 1e-11 * abs(E1), i
        else:
            assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b), i
            assert abs(E - E1) <= 1e-5 * abs(E1), i
    # A second launch of the cached graph gives the same results.
    T0 = [t.clone() for t in T]
    for t in T:
        t.zero_()
    c.gw_solve_batch(probs, u, v, T, st, phi, psi)
    c.gw_ctx_check()
    assert all(torch.equal(a, b) for a, b in zip(T0, T))


def test_batch_fp64_matches_oracle():
    from paper_2404_08970_gb300 import _lib as L
    ws = [w for w in _mixed() if w.get("dim", 1) == 1 and w.get("phi") is None and w["nx"] * w["ny"] <= 400000]
    c = U.ctx()
    probs = [_prob(L, w, "f64") for w in ws]
    u, v, T, st, phi, psi = _dev(ws, "f64")
    c.gw_solve_batch(probs, u, v, T, st)
    c.gw_ctx_check()
    for i, w in enumerate(ws):
        DX, DY = O.grid_dist_1d(w["nx"], w["hx"], w["k"]), O.grid_dist_1d(w["ny"], w["hy"], w["k"])
        Ts, _, _ = O.mirror_descent(DX, DY, w["u"], w["v"], w["eps"], w["n_outer"], w["n_inner"], tau=w.get("tau"),
                                    warm_start=bool(w.get("warm", 0)))
        assert U.relerr(T[i].cpu().numpy(), Ts) < 1e-9, i


def test_batch_rejects_bad_problem():
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    u = torch.full((4,), 0.25, dtype=torch.float64, device="cuda")
    T = torch.empty(4, 4, device="cuda")
    good = L.problem(dim=1, nx=4, ny=4, eps=0.1, n_outer=1, n_inner=1)
    bad = L.problem(dim=1, nx=4, ny=4, eps=-1.0, n_outer=1, n_inner=1)
    with pytest.raises(L.GWError) as e:
        c.gw_solve_batch([good, bad], [u, u], [u, u], [T, T])
    assert e.value.status == L.GW_ERR_INVALID
    assert "[1]" in str(e.value)
    c.gw_solve_batch([], [], [], [])



def test_batch_mixed_and_grouped_problems():
    """Problems whose row configuration runs 512-thread blocks share every
    Sinkhorn launch (one launch per pass over all of them, each block running
    its own problem's configuration); longer rows (here 9000 columns) run in
    their own group beside them.  Every result equals the single solve."""
    import torch
    from paper_2404_08970_gb300 import _lib as L
    rng = np.random.default_rng(8)
    shapes = [(40, 9000, 1), (300, 257, 2), (129, 3001, 1), (700, 75, 1), (64, 8192, 2), (33, 4097, 1)]
    ws = [dict(nx=n, ny=m, hx=1.0 / n, hy=1.0 / m, k=k, eps=5e-2, n_outer=2, n_inner=20,
               u=I.dirichlet(n, 1.0, rng), v=I.dirichlet(m, 1.0, rng)) for (n, m, k) in shapes]
    c = U.ctx()
    probs = [_prob(L, w, "f32") for w in ws]
    u, v, T, st, phi, psi = _dev(ws, "f32")
    c.gw_solve_batch(probs, u, v, T, st)
    c.gw_ctx_check()
    for i, w in enumerate(ws):
        T1 = torch.empty_like(T[i])
        s1 = torch.zeros(8, dtype=torch.float64, device="cuda")
        c.gw_solve(probs[i], u[i], v[i], T1, None, None, s1)
        c.gw_ctx_check()
        a, b = T[i].double().cpu().numpy(), T1.double().cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b), i
        assert abs(float(st[i][0]) - float(s1[0])) <= 1e-5 * abs(float(s1[0])), i
        assert float(st[i][5]) < 1e-5, i

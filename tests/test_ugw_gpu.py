"""Entropic unbalanced GW (Remark "Entropic algorithm for UGW") on the GPU,
through gw_solve with prob->rho > 0, against the FP64 oracle's ugw_solve
(same schedule: T^0 = u v^T / sqrt(m(u) m(v)), each step the unbalanced
Sinkhorn iteration on the cost ((1/2) grad E + g) / m from f = g = 0, then
the mass rescale).  Marginals of unequal masses.  Tolerances as for the
balanced solve: double 1e-9 (plan) and 1e-10 (values), float 1e-5 on the
UGW objective."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2404_08970_gb300 import inputs as I
from tests import gwtest_util as U

pytestmark = pytest.mark.gpu


def _prob(L, w, dtype):
    return L.problem(dim=w.get("dim", 1), nx=w["nx"], ny=w["ny"], hx=w["hx"], hy=w["hy"], k=w["k"],
                     cost=w.get("cost", 0), eps=w["eps"], n_outer=w["n_outer"], n_inner=w["n_inner"],
                     dtype=L.GW_F32 if dtype == "f32" else L.GW_F64, rho=w["rho"],
                     warm_start=w.get("warm", 0))


def gpu_ugw(w, dtype):
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    n = w["nx"] ** 2 if w.get("dim", 1) == 2 else w["nx"]
    m = w["ny"] ** 2 if w.get("dim", 1) == 2 else w["ny"]
    T = torch.empty(n, m, dtype=torch.float32 if dtype == "f32" else torch.float64, device="cuda")
    st = torch.zeros(8, dtype=torch.float64, device="cuda")
    c.gw_solve(_prob(L, w, dtype), torch.from_numpy(w["u"]).cuda(), torch.from_numpy(w["v"]).cuda(), T, None, None,
               st)
    c.gw_ctx_check()
    return T.double().cpu().numpy(), st.cpu().numpy()


def oracle_ugw(w):
    if w.get("dim", 1) == 2:
        DX = O.grid_dist_2d(w["nx"], w["hx"], "sqeuclid")
        DY = O.grid_dist_2d(w["ny"], w["hy"], "sqeuclid")
    else:
        DX, DY = O.grid_dist_1d(w["nx"], w["hx"], w["k"]), O.grid_dist_1d(w["ny"], w["hy"], w["k"])
    T, _, _ = O.ugw_solve(DX, DY, w["u"], w["v"], w["eps"], w["rho"], w["n_outer"], w["n_inner"])
    return T, dict(obj=O.ugw_value(DX, DY, T, w["u"], w["v"], w["rho"], w["eps"]), E=O.value(DX, DY, T),
                   mass=float(T.sum()))


def _w1d(n, m, k, rho, seed, mu=1.3, mv=0.8):
    rng = np.random.default_rng(seed)
    return dict(nx=n, ny=m, hx=1.0 / n, hy=1.0 / m, k=k, eps=5e-2, n_outer=5, n_inner=40, rho=rho,
                u=I.dirichlet(n, 1.0, rng) * mu, v=I.dirichlet(m, 1.0, rng) * mv)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shape,k,rho", [((9, 7), 1, 0.5), ((64, 150), 1, 1.0), ((150, 64), 2, 0.2),
                                         ((33, 1000), 1, 5.0)])
def test_ugw_1d_matches_oracle(shape, k, rho, dtype):
    w = _w1d(*shape, k, rho, seed=shape[0] + 3 * shape[1])
    T, st = gpu_ugw(w, dtype)
    Ts, ss = oracle_ugw(w)
    if dtype == "f64":
        assert U.relerr(T, Ts) < 1e-9, U.relerr(T, Ts)
        assert abs(st[0] - ss["obj"]) <= 1e-10 * abs(ss["obj"])
        assert abs(st[1] - ss["E"]) <= 1e-10 * abs(ss["E"])
        assert abs(st[7] - ss["mass"]) <= 1e-12 * ss["mass"]
    else:
        assert abs(st[0] - ss["obj"]) <= 1e-5 * abs(ss["obj"]), (st[0], ss["obj"])
        assert np.linalg.norm(T - Ts) <= 1e-3 * np.linalg.norm(Ts)
        assert abs(st[7] - ss["mass"]) <= 1e-5 * ss["mass"]


def test_ugw_2d_matches_oracle():
    rng = I.rng_for(81)
    w = dict(dim=2, cost=1, nx=6, ny=8, hx=0.2, hy=1 / 7, k=1, eps=5e-2, n_outer=4, n_inner=40, rho=0.5,
             u=I.abs_normal_image(6, rng) * 1.2, v=I.abs_normal_image(8, rng) * 0.9)
    T, st = gpu_ugw(w, "f64")
    Ts, ss = oracle_ugw(w)
    assert U.relerr(T, Ts) < 1e-9
    assert abs(st[0] - ss["obj"]) <= 1e-10 * abs(ss["obj"])


def test_ugw_large_rho_is_balanced_gw_on_the_gpu():
    """rho -> infinity with unit masses: the GPU UGW plan is the balanced
    solve's with the cost halved (balanced gw_solve at 2 eps)."""
    import torch
    from paper_2404_08970_gb300 import _lib as L
    w = _w1d(40, 30, 1, 1e7, seed=82, mu=1.0, mv=1.0)
    T, st = gpu_ugw(w, "f64")
    c = U.ctx()
    Tb = torch.empty(40, 30, dtype=torch.float64, device="cuda")
    pb = L.problem(dim=1, nx=40, ny=30, hx=w["hx"], hy=w["hy"], k=1, eps=2 * w["eps"], n_outer=w["n_outer"],
                   n_inner=w["n_inner"], dtype=L.GW_F64)
    c.gw_solve(pb, torch.from_numpy(w["u"]).cuda(), torch.from_numpy(w["v"]).cuda(), Tb)
    c.gw_ctx_check()
    assert U.relerr(T, Tb.cpu().numpy()) < 1e-6


def test_ugw_batch_equals_single():
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    ws = [_w1d(50, 70, 1, 0.5, seed=83), _w1d(90, 40, 2, 2.0, seed=84)]
    probs = [_prob(L, w, "f64") for w in ws]
    u = [torch.from_numpy(w["u"]).cuda() for w in ws]
    v = [torch.from_numpy(w["v"]).cuda() for w in ws]
    T = [torch.empty(w["nx"], w["ny"], dtype=torch.float64, device="cuda") for w in ws]
    st = [torch.zeros(8, dtype=torch.float64, device="cuda") for _ in ws]
    c.gw_solve_batch(probs, u, v, T, st)
    c.gw_ctx_check()
    for i, w in enumerate(ws):
        T1, s1 = gpu_ugw(w, "f64")
        assert U.relerr(T[i].cpu().numpy(), T1) < 1e-11
        assert abs(float(st[i][0]) - s1[0]) <= 1e-11 * abs(s1[0])


def test_ugw_rejects_fused_and_tau():
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    u = torch.full((4,), 0.25, dtype=torch.float64, device="cuda")
    T = torch.empty(4, 4, device="cuda")
    for kw in (dict(rho=-1.0), dict(rho=0.5, tau=0.2), dict(rho=0.5, theta=0.5, feat_dim=2)):
        p = L.problem(dim=1, nx=4, ny=4, eps=0.1, n_outer=1, n_inner=1, **kw)
        with pytest.raises(L.GWError) as e:
            c.gw_solve(p, u, u, T, phi=u.view(4, 1).repeat(1, 2).contiguous(), psi=u.view(4, 1).repeat(1, 2).contiguous())
        assert e.value.status == L.GW_ERR_INVALID

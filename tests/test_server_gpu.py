"""The request server (gw_server_*): results equal gw_solve on the same
inputs (same launch sequence and row bands, so bit for bit), admission under
a memory budget, and error reporting."""
import time

import numpy as np
import pytest

from paper_2404_08970_gb300 import inputs as I
from tests import gwtest_util as U

pytestmark = pytest.mark.gpu


def _prob(L, r, dtype):
    return L.problem(dim=r["dim"], nx=r["nx"], ny=r["ny"], hx=r["hx"], hy=r["hy"], k=r["k"],
                     cost=L.GW_COST_SQEUCLID if r.get("cost") == "sqeuclid" else L.GW_COST_POW, eps=r["eps"],
                     n_outer=r["n_outer"], n_inner=r["n_inner"], theta=r["theta"],
                     feat_dim=0 if r.get("phi") is None else r["phi"].shape[1], dtype=dtype)


def _wait(srv, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                res = srv.poll(t)
                if res is not None:
                    out[t] = res
        assert time.time() - t0 < timeout, "requests did not finish"
        time.sleep(0.002)
    return out


def _direct(L, r, dtype):
    import torch
    c = U.ctx()
    n = r["nx"] ** 2 if r["dim"] == 2 else r["nx"]
    m = r["ny"] ** 2 if r["dim"] == 2 else r["ny"]
    tdt = torch.float32 if dtype == L.GW_F32 else torch.float64
    T = torch.empty(n, m, dtype=tdt, device="cuda")
    st = torch.zeros(8, dtype=torch.float64, device="cuda")
    phi = None if r.get("phi") is None else torch.from_numpy(r["phi"]).cuda()
    psi = None if r.get("psi") is None else torch.from_numpy(r["psi"]).cuda()
    c.gw_solve(_prob(L, r, dtype), torch.from_numpy(r["u"]).cuda(), torch.from_numpy(r["v"]).cuda(), T, None, None,
               st, phi, psi)
    c.gw_ctx_check()
    return T.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("dtype_name", ["f32", "f64"])
def test_server_matches_gw_solve(dtype_name):
    from paper_2404_08970_gb300 import _lib as L
    dtype = L.GW_F32 if dtype_name == "f32" else L.GW_F64
    reqs = I.workload_serve(8, rate=1000.0, seed=3, lo=64, hi=900, n_outer=3, n_inner=20)
    srv = L.Server(0, hbm_budget_bytes=2 << 30, max_slots=3)
    try:
        outs, tickets = [], []
        for r in reqs:
            n = r["nx"] ** 2 if r["dim"] == 2 else r["nx"]
            m = r["ny"] ** 2 if r["dim"] == 2 else r["ny"]
            T = np.empty((n, m), dtype=np.float32 if dtype == L.GW_F32 else np.float64)
            outs.append(T)
            tickets.append(srv.submit(_prob(L, r, dtype), r["u"], r["v"], r.get("phi"), r.get("psi"), T))
        res = _wait(srv, tickets)
        for r, t, T in zip(reqs, tickets, outs):
            st, stats, lat = res[t]
            assert st == L.GW_OK and lat > 0, srv.last_error()
            Td, sd = _direct(L, r, dtype)
            assert np.array_equal(T, Td), r["kind"]
            assert np.array_equal(np.array(stats), sd), r["kind"]
        assert srv.info()[0] == 0
    finally:
        srv.close()


def test_server_budget_admission_and_errors():
    from paper_2404_08970_gb300 import _lib as L
    reqs = I.workload_serve(6, rate=1000.0, seed=5, lo=200, hi=400, n_outer=2, n_inner=10)
    # A budget that holds about one request at a time: everything still finishes.
    srv = L.Server(0, hbm_budget_bytes=24 << 20, max_slots=4)
    try:
        tickets = [srv.submit(_prob(L, r, L.GW_F32), r["u"], r["v"], r.get("phi"), r.get("psi")) for r in reqs]
        res = _wait(srv, tickets)
        assert all(v[0] == L.GW_OK for v in res.values())
        # Reported once; unknown tickets are invalid.
        with pytest.raises(L.GWError):
            srv.poll(tickets[0])
        # Larger than the budget: rejected at submission.
        big = dict(reqs[0], dim=1, nx=16384, ny=16384, hx=1 / 16384, hy=1 / 16384, theta=1.0, phi=None, psi=None,
                   u=I.uniform_weights(16384), v=I.uniform_weights(16384), kind="1d")
        with pytest.raises(L.GWError) as e:
            srv.submit(_prob(L, big, L.GW_F32), big["u"], big["v"])
        assert e.value.status == L.GW_ERR_INVALID
        bad = dict(reqs[0], eps=-1.0)
        with pytest.raises(L.GWError):
            srv.submit(_prob(L, bad, L.GW_F32), bad["u"], bad["v"], bad.get("phi"), bad.get("psi"))
    finally:
        srv.close()


def test_server_shutdown_with_queued_requests():
    from paper_2404_08970_gb300 import _lib as L
    reqs = I.workload_serve(20, rate=1000.0, seed=6, lo=500, hi=2000, n_outer=2, n_inner=20)
    srv = L.Server(0, hbm_budget_bytes=1 << 30, max_slots=1)
    for r in reqs:
        srv.submit(_prob(L, r, L.GW_F32), r["u"], r["v"], r.get("phi"), r.get("psi"))
    srv.close()  # running request finishes, the queued ones end with GW_ERR_SHUTDOWN


def test_server_small_requests_pass_a_waiting_large_one():
    """Two large requests that cannot run together under the budget, then
    small ones: the small ones run beside the first large request instead of
    queueing behind the second (no head-of-line blocking), and the second
    large request still finishes."""
    from paper_2404_08970_gb300 import _lib as L
    rng = np.random.default_rng(8)

    def req(n, n_outer, n_inner):
        return dict(dim=1, nx=n, ny=n, hx=1.0 / n, hy=1.0 / n, k=1, eps=5e-2, n_outer=n_outer, n_inner=n_inner,
                    theta=1.0, u=I.dirichlet(n, 1.0, rng), v=I.dirichlet(n, 1.0, rng))

    big = [req(4096, 10, 50), req(4096, 10, 50)]   # about 140 MB each while running
    small = [req(200, 3, 20) for _ in range(4)]      # well under 1 MB each
    srv = L.Server(0, hbm_budget_bytes=200 << 20, max_slots=4)
    try:
        tb = [srv.submit(_prob(L, r, L.GW_F32), r["u"], r["v"]) for r in big]
        ts = [srv.submit(_prob(L, r, L.GW_F32), r["u"], r["v"]) for r in small]
        res = _wait(srv, tb + ts)
        assert all(v[0] == L.GW_OK for v in res.values()), srv.last_error()
        lat_b2 = res[tb[1]][2]
        assert max(res[t][2] for t in ts) < lat_b2, ([res[t][2] for t in ts], lat_b2)
    finally:
        srv.close()

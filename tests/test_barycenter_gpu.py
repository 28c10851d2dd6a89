"""Parity of the fixed-support GW barycenter (CUDA, through the C ABI) with
the FP64 oracle's barycenter iteration: entropic GW solves between the dense
barycenter (C, p) and each 1D grid input by mirror descent, then the
square-loss update C = sum_s lambda_s T_s D_s T_s^T / (sum lambda p p^T).

Tolerances: double reproduces the oracle's C to 1e-9 (max relative error);
float to 2e-4, the plans' float error carried through the update."""
import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2404_08970_gb300 import inputs as I
from tests import gwtest_util as U

pytestmark = pytest.mark.gpu


def _case(N, ns, k, seed):
    rng = np.random.default_rng(seed)
    hs = [1.0 / n for n in ns]
    ps = [I.dirichlet(n, 1.0, rng) for n in ns]
    p = I.dirichlet(N, 2.0, rng)
    lam = list(rng.uniform(0.2, 1.0, len(ns)))
    C0 = rng.uniform(0.0, 0.5, (N, N))
    C0 = (C0 + C0.T) / 2
    np.fill_diagonal(C0, 0.0)
    return hs, ps, p, lam, C0


def gpu_barycenter(N, ns, k, hs, ps, p, lam, C0, eps, n_iter, n_outer, n_inner, dtype):
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    tdt = torch.float32 if dtype == "f32" else torch.float64
    dC = torch.from_numpy(C0).to("cuda", tdt)
    dps = [torch.from_numpy(q).cuda() for q in ps]
    dp = torch.from_numpy(p).cuda()
    stats = torch.zeros(8 * len(ns), dtype=torch.float64, device="cuda")
    prob = L.gw_barycenter_problem(len(ns), N, k, L.GW_F32 if dtype == "f32" else L.GW_F64, eps, n_iter, n_outer,
                                   n_inner)
    c.gw_barycenter(prob, ns, hs, lam, dps, dp, dC, stats)
    c.gw_ctx_check()
    return dC.double().cpu().numpy(), stats.cpu().numpy().reshape(len(ns), 8)


def oracle_barycenter(N, ns, k, hs, ps, p, lam, C0, eps, n_iter, n_outer, n_inner):
    Cs = [O.grid_dist_1d(n, h, k) for n, h in zip(ns, hs)]
    return O.barycenter(Cs, ps, lam, p, C0, eps, n_iter, n_outer, n_inner)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("N,ns,k", [(12, (15, 20, 9), 1), (20, (33, 64), 2), (7, (100,), 1), (65, (70, 31), 2),
                                    (300, (700,), 1)])
def test_barycenter_matches_oracle(N, ns, k, dtype):
    hs, ps, p, lam, C0 = _case(N, ns, k, seed=N + sum(ns))
    args = (N, ns, k, hs, ps, p, lam, C0, 5e-2, 3, 4, 40)
    C, st = gpu_barycenter(*args, dtype)
    Cs, Ts = oracle_barycenter(*args)
    tol = 1e-9 if dtype == "f64" else 2e-4
    assert U.relerr(C, Cs) < tol, U.relerr(C, Cs)
    assert np.max(np.abs(C - C.T)) <= 1e-6 * np.max(np.abs(C))
    # The statistics of the last round's solves: E against the C of that
    # round (the oracle's couplings are those solves' plans).
    assert np.all(np.isfinite(st)) and np.all(st[:, 1] >= 0.0)


def test_barycenter_graph_relaunch_is_identical():
    import torch
    N, ns, k = 16, (24, 40), 1
    hs, ps, p, lam, C0 = _case(N, ns, k, seed=2)
    a, _ = gpu_barycenter(N, ns, k, hs, ps, p, lam, C0, 5e-2, 2, 3, 30, "f32")
    b, _ = gpu_barycenter(N, ns, k, hs, ps, p, lam, C0, 5e-2, 2, 3, 30, "f32")
    assert np.array_equal(a, b)


@pytest.mark.parametrize("bad", ["count", "k", "N", "lambda", "h"])
def test_barycenter_rejects_bad_arguments(bad):
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    N, ns = 4, [5]
    hs, lam = [0.2], [1.0]
    prob = L.gw_barycenter_problem(1, N, 1, L.GW_F32, 0.1, 1, 1, 1)
    if bad == "count":
        prob.count = 0
    elif bad == "k":
        prob.k = 3
    elif bad == "N":
        prob.N = 0
    elif bad == "lambda":
        lam = [-1.0]
    else:
        hs = [float("inf")]
    dC = torch.zeros(N, N, device="cuda")
    dp = torch.full((N,), 0.25, dtype=torch.float64, device="cuda")
    dps = [torch.full((5,), 0.2, dtype=torch.float64, device="cuda")]
    with pytest.raises(L.GWError) as e:
        c.gw_barycenter(prob, ns, hs, lam, dps, dp, dC)
    assert e.value.status == L.GW_ERR_INVALID

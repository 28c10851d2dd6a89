"""The seeded workload generators: shapes, ranges and determinism (CPU)."""
import numpy as np

from paper_2404_08970_gb300 import inputs as I


def test_batch_workload_generator():
    ws = I.workload_batch(256, seed=0)
    assert len(ws) == 256
    ns = np.array([w["nx"] for w in ws] + [w["ny"] for w in ws])
    assert ns.min() >= 256 and ns.max() <= 8192
    # log-uniform: about half the sizes below the geometric midpoint 1448
    assert 0.4 < np.mean(ns < 1448) < 0.6
    assert set(w["k"] for w in ws) == {1, 2}
    for w in ws[:5]:
        assert abs(w["u"].sum() - 1) < 1e-12 and abs(w["v"].sum() - 1) < 1e-12
    again = I.workload_batch(256, seed=0)
    assert [(w["nx"], w["ny"], w["k"]) for w in ws] == [(w["nx"], w["ny"], w["k"]) for w in again]


def test_random_coupling_is_positive_with_marginals():
    rng = I.rng_for(0)
    u, v = I.dirichlet(30, 0.5, rng), I.dirichlet(40, 0.5, rng)
    T = I.random_coupling(u, v, rng)
    assert np.all(T > 0)
    assert np.max(np.abs(T.sum(1) - u)) < 1e-15 and np.max(np.abs(T.sum(0) - v)) < 1e-15


def test_serve_workload_generator():
    reqs = I.workload_serve(400, rate=2000.0, seed=0)
    kinds = [r["kind"] for r in reqs]
    for k in I.SERVE_KINDS:
        assert 0.15 < kinds.count(k) / len(kinds) < 0.35
    gaps = np.diff([0.0] + [r["arrival"] for r in reqs])
    assert np.all(gaps > 0) and 0.5 / 2000 < gaps.mean() < 1.5 / 2000
    for r in reqs:
        n = r["nx"] ** 2 if r["dim"] == 2 else r["nx"]
        m = r["ny"] ** 2 if r["dim"] == 2 else r["ny"]
        assert 100 <= n <= 16384 + 300 and 100 <= m <= 16384 + 300
        assert abs(r["u"].sum() - 1) < 1e-12 and r["u"].size == n
        if r["kind"].endswith("fgw"):
            assert r["phi"].shape == (n, 16) and r["psi"].shape == (m, 16) and r["theta"] == 0.5


def test_volume_workload_generator():
    w = I.workload_3d(6, 7, "manhattan", seed=0)
    assert w["dim"] == 3 and w["u"].shape == (216,) and w["v"].shape == (343,)
    assert np.all(w["u"] > 0) and abs(w["u"].sum() - 1) < 1e-12 and abs(w["v"].sum() - 1) < 1e-12
    assert w["hx"] == 1.0 / 5 and w["hy"] == 1.0 / 6
    again = I.workload_3d(6, 7, "manhattan", seed=0)
    assert np.array_equal(w["u"], again["u"])

"""Every Sinkhorn row configuration the tuning table can select runs and
gives the oracle's result.  For each row length, every candidate that is not
the built-in choice is installed for exactly that row length (gw_tune_set),
a small solve runs under it, and its plan and value are compared with the
FP64 oracle's mirror descent and with the solve under the built-in choice."""
import os

import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2404_08970_gb300 import inputs as I
from tests import gwtest_util as U

pytestmark = pytest.mark.gpu

ROWS = {"f32": [300, 700, 1000, 1500, 2000, 3000, 4000, 6000, 8000, 10000], "f64": [200, 1000, 4000]}
TABLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2404_08970_gb300",
                     "tune_table.txt")


def _reload_committed_table(L):
    """The table the library loads at start-up (beside the library)."""
    if os.path.exists(TABLE):
        L.gw_tune_load(TABLE)


def _table_entries():
    out = []
    for line in open(TABLE):
        body = line.split("#")[0].split()
        if len(body) == 5:
            out.append(tuple(int(x) for x in body))
    return out


def test_committed_table_is_in_effect_and_solves_match_oracle():
    """The committed tuning table is loaded at context creation; a solve in
    each tuned range runs under the table's configuration and matches the
    FP64 oracle."""
    from paper_2404_08970_gb300 import _lib as L
    U.ctx()
    L.gw_tune_clear()
    _reload_committed_table(L)
    entries = _table_entries()
    assert entries
    for kernel, dt, lo, hi, cfg in entries:
        assert L.gw_tune_config(kernel, dt, hi) == cfg
    for kernel, dt, lo, hi, cfg in entries:
        if dt != L.GW_F32 or hi > 4096 or cfg == L.gw_tune_candidates(kernel, dt, hi)[0]:
            continue
        m = hi
        rng = np.random.default_rng(m + 1)
        n = 16
        w = dict(nx=n, ny=m, hx=1.0 / n, hy=1.0 / m, k=1, eps=5e-2, n_outer=3, n_inner=30,
                 u=I.dirichlet(n, 1.0, rng), v=I.dirichlet(m, 1.0, rng))
        DX, DY = O.grid_dist_1d(n, w["hx"], 1), O.grid_dist_1d(m, w["hy"], 1)
        Ts, _, _ = O.mirror_descent(DX, DY, w["u"], w["v"], w["eps"], w["n_outer"], w["n_inner"])
        T, st = _solve(w, "f32")
        assert np.linalg.norm(T - Ts) <= 1e-3 * np.linalg.norm(Ts), (m, cfg)
        assert abs(st[1] - O.value(DX, DY, Ts)) <= 1e-5 * O.value(DX, DY, Ts), (m, cfg)


def _solve(w, dtype):
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    n, m = w["nx"], w["ny"]
    T = torch.empty(n, m, dtype=torch.float32 if dtype == "f32" else torch.float64, device="cuda")
    st = torch.zeros(8, dtype=torch.float64, device="cuda")
    prob = L.problem(dim=1, nx=n, ny=m, hx=w["hx"], hy=w["hy"], k=w["k"], eps=w["eps"], n_outer=w["n_outer"],
                     n_inner=w["n_inner"], dtype=L.GW_F32 if dtype == "f32" else L.GW_F64)
    c.gw_solve(prob, torch.from_numpy(w["u"]).cuda(), torch.from_numpy(w["v"]).cuda(), T, None, None, st)
    c.gw_ctx_check()
    return T.double().cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_every_alternative_configuration_matches_oracle(dtype):
    from paper_2404_08970_gb300 import _lib as L
    SK = L.GW_TUNE_SINKHORN
    dt = L.GW_F32 if dtype == "f32" else L.GW_F64
    L.gw_tune_clear()
    seen = set()
    try:
        for m in ROWS[dtype]:
            rng = np.random.default_rng(m)
            n, k = 24, 1 + m % 2
            w = dict(nx=n, ny=m, hx=1.0 / n, hy=1.0 / m, k=k, eps=5e-2, n_outer=3, n_inner=30,
                     u=I.dirichlet(n, 1.0, rng), v=I.dirichlet(m, 1.0, rng))
            DX, DY = O.grid_dist_1d(n, w["hx"], k), O.grid_dist_1d(m, w["hy"], k)
            Ts, _, _ = O.mirror_descent(DX, DY, w["u"], w["v"], w["eps"], w["n_outer"], w["n_inner"])
            Es = O.value(DX, DY, Ts)
            base = L.gw_tune_config(SK, dt, m)
            Tb, sb = _solve(w, dtype)
            seen.add(base)
            if dtype == "f32":
                assert np.linalg.norm(Tb - Ts) <= 1e-3 * np.linalg.norm(Ts), (m, base)
                assert abs(sb[1] - Es) <= 1e-5 * abs(Es), (m, base, sb[1], Es)
            for cfg in L.gw_tune_candidates(SK, dt, m)[1:]:
                L.gw_tune_set(SK, dt, m, m, cfg)
                assert L.gw_tune_config(SK, dt, m) == cfg
                T, st = _solve(w, dtype)
                L.gw_tune_clear()
                seen.add(cfg)
                if dtype == "f64":
                    assert U.relerr(T, Ts) < 1e-9, (m, cfg)
                    assert U.relerr(T, Tb) < 1e-11, (m, cfg, base)
                    assert abs(st[1] - Es) <= 1e-10 * abs(Es), (m, cfg)
                else:
                    assert np.linalg.norm(T - Ts) <= 1e-3 * np.linalg.norm(Ts), (m, cfg)
                    assert abs(st[1] - Es) <= 1e-5 * abs(Es), (m, cfg, st[1], Es)
                    assert st[5] < 1e-5, (m, cfg)
    finally:
        L.gw_tune_clear()
        _reload_committed_table(L)
    # Every configuration of this dtype up to 16384 columns ran at least once
    # (as the built-in choice or as an alternative).
    alts = set(range(0, 7)) | set(range(20, 25)) | set(range(40, 49)) | set(range(50, 56)) if dtype == "f32" \
        else {30, 31, 32}
    assert alts <= seen, alts - seen

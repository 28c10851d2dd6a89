"""The dense comparison gradient (cuBLAS) against the FP64 oracle.  FP64 and
FP32 are exact up to their rounding; TF32 and BF16 errors are measured and
bounded loosely (they are the stated reduced-precision forms)."""
import numpy as np
import pytest

from paper_2404_08970_gb300 import inputs as I
from tests import gwtest_util as U

pytestmark = pytest.mark.gpu

BOUND = {"fp64": 1e-12, "fp32": 1e-5, "tf32": 2e-2, "bf16": 1e-1}


def gpu_dense(T, u, v, k, hx, hy, prec, marginals="target"):
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = U.ctx()
    tdt = torch.float64 if prec == "fp64" else torch.float32
    dT = torch.from_numpy(np.ascontiguousarray(T)).to("cuda", tdt)
    dG = torch.empty_like(dT)
    n, m = T.shape
    prob = L.problem(dim=1, nx=n, ny=m, hx=hx, hy=hy, k=k, dtype=L.GW_F64 if prec == "fp64" else L.GW_F32)
    P = {"fp32": L.GW_DENSE_FP32, "tf32": L.GW_DENSE_TF32, "bf16": L.GW_DENSE_BF16, "fp64": L.GW_DENSE_FP64}[prec]
    mg = L.GW_MARG_TARGET if marginals == "target" else L.GW_MARG_EXACT
    c.gw_grad_dense(prob, torch.from_numpy(u).cuda() if u is not None else None,
                    torch.from_numpy(v).cuda() if v is not None else None, dT, dG, mg, P)
    c.gw_ctx_check()
    return dG.double().cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("shape", [(64, 48), (300, 257), (1024, 1024)], ids=lambda s: f"{s[0]}x{s[1]}")
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

"""Shared helpers for the GPU parity tests: run the CUDA path through the
C ABI and the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

from oracle import gw_oracle as O


def relerr(a, b) -> float:
    """max |a - b| / max |b| (the gradient's relative error)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


_CTX = None


def ctx():
    global _CTX
    if _CTX is None:
        import __graft_entry__
        __graft_entry__.build()
        from paper_2404_08970_gb300 import _lib as L
        _CTX = L.Context(0)
    return _CTX


def gpu_grad_1d(T: np.ndarray, u, v, k: int, hx: float, hy: float, dtype: str, marginals: str):
    """Runs gw_grad on the GPU; T is already in the compute dtype."""
    import torch
    from paper_2404_08970_gb300 import _lib as L
    c = ctx()
    n, m = T.shape
    tdt = torch.float32 if dtype == "f32" else torch.float64
    dT = torch.from_numpy(np.ascontiguousarray(T)).to("cuda", tdt)
    dG = torch.empty_like(dT)
    du = torch.from_numpy(np.asarray(u, dtype=np.float64)).cuda() if u is not None else None
    dv = torch.from_numpy(np.asarray(v, dtype=np.float64)).cuda() if v is not None else None
    prob = L.problem(dim=1, nx=n, ny=m, hx=hx, hy=hy, k=k, dtype=L.GW_F32 if dtype == "f32" else L.GW_F64)
    mg = L.GW_MARG_TARGET if marginals == "target" else L.GW_MARG_EXACT
    c.gw_grad(prob, du, dv, dT, dG, mg)
    c.gw_ctx_check()
    return dG.double().cpu().numpy()


def oracle_grad_1d(T64: np.ndarray, u, v, k: int, hx: float, hy: float, marginals: str):
    n, m = T64.shape
    DX, DY = O.grid_dist_1d(n, hx, k), O.grid_dist_1d(m, hy, k)
    if marginals == "target":
        return O.grad(DX, DY, T64, np.asarray(u), np.asarray(v))
    return O.grad_exact(DX, DY, T64)


def oracle_grad_rows_1d(T64: np.ndarray, rows, u, v, k: int, hx: float, hy: float):
    """Rows `rows` of the oracle gradient with target marginals, without
    forming D_X in full."""
    n, m = T64.shape
    idx = np.arange(n, dtype=np.float64)
    rows = np.asarray(rows)
    DXr = (hx ** k) * np.abs(idx[rows][:, None] - idx[None, :]) ** k
    DY = O.grid_dist_1d(m, hy, k)
    cx_rows = (DXr * DXr) @ np.asarray(u)
    cy = (DY * DY) @ np.asarray(v)
    return O.grad_rows(DXr, DY, T64, cx_rows, cy)

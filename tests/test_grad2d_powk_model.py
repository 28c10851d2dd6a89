"""Precision model of the 2D Manhattan^k gradient for k >= 2 (Sec. 3.1, eqs.
"2d Dx", "2d gradient", "2D kronecker"), checked against the FP64 oracle on
the CPU.

The GPU path transforms each row of T as an sy x sy image, then each column
of the result as an sx x sx image, with

    D-hat = sum_s C(k, s) A_{k-s} (x) A_s,   A_j = |i - j|^j,  A_0 = J,

where each line transform A_j x is one forward and one backward pass of the
recursion over the states F_s(i) = sum_{j<i} (i - j)^s x_j (s = 0..k, all
non-negative, no cancellation).  The two end terms (s = 0 and s = k) reduce
to 1D transforms of the image's row and column sums; the k - 1 middle terms
transform the whole image along both axes.  This file re-states that
arithmetic in numpy, in float32 for every operation the kernels do in float,
and checks that (a) in float64 it reproduces the oracle's dense definition
to rounding and (b) in float32 it stays within the 1e-6 gradient bound, so
that plain float scans suffice.  The reference is always the oracle.
"""
import math

import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2404_08970_gb300 import inputs as I


def line_transforms(x, k, dt):
    """A_s x along the last axis for s = 0..k (A_0 = J), by the forward and
    backward recursions in dtype dt.  x: (..., L)."""
    x = x.astype(dt)
    L = x.shape[-1]
    fwd = np.zeros((k + 1,) + x.shape, dtype=dt)
    st = np.zeros((k + 1,) + x.shape[:-1], dtype=dt)
    for i in range(L):
        for s in range(k + 1):
            fwd[s, ..., i] = st[s]
        # S_s(i+1) = sum_u C(s,u) S_u(i) + x_i   (binomial expansion of (i+1-j)^s)
        new = np.empty_like(st)
        for s in range(k + 1):
            acc = x[..., i].copy()
            for u in range(s + 1):
                acc = (acc + dt(math.comb(s, u)) * st[u]).astype(dt)
            new[s] = acc
        st = new
    bwd = np.zeros_like(fwd)
    st = np.zeros((k + 1,) + x.shape[:-1], dtype=dt)
    for i in range(L - 1, -1, -1):
        for s in range(k + 1):
            bwd[s, ..., i] = st[s]
        new = np.empty_like(st)
        for s in range(k + 1):
            acc = x[..., i].copy()
            for u in range(s + 1):
                acc = (acc + dt(math.comb(s, u)) * st[u]).astype(dt)
            new[s] = acc
        st = new
    out = (fwd + bwd).astype(dt)
    out[0] = (out[0] + x).astype(dt)  # A_0 = J includes the diagonal
    return out


def image_transform(Y, k, dt):
    """sum_s C(k,s) A_{k-s} (along axis -2) Y A_s (along axis -1) for images
    Y (..., L, L), computed as the kernels do."""
    Y = Y.astype(dt)
    L = Y.shape[-1]
    rs = Y.sum(axis=-1, dtype=dt)                        # row sums (over d)
    cs = Y.sum(axis=-2, dtype=dt)                        # column sums (over c)
    e0 = line_transforms(rs, k, dt)[k]                   # A_k (Y 1), along c
    ek = line_transforms(cs, k, dt)[k]                   # A_k (1^T Y), along d
    R = line_transforms(Y, k - 1, dt)                    # A_s along d, s < k
    W = (e0[..., :, None] + ek[..., None, :]).astype(dt)
    for s in range(1, k):
        Cs = line_transforms(np.swapaxes(R[s], -1, -2), k - s, dt)[k - s]  # A_{k-s} along c
        W = (W + dt(math.comb(k, s)) * np.swapaxes(Cs, -1, -2)).astype(dt)
    return W


def model_grad(T, sx, sy, hx, hy, k, u, v, dt):
    """G = c_x + c_y - 2 D_X T D_Y: rows as Y images, then columns as X
    images, then the epilogue with constant terms computed in float64 (the
    kernels compute them in double and round once)."""
    n, m = T.shape
    W = image_transform(T.reshape(n, sy, sy), k, dt).reshape(n, m)
    Z = image_transform(W.T.reshape(m, sx, sx), k, dt).reshape(m, n).T
    DX = O.grid_dist_2d(sx, hx, "manhattan", k)
    DY = O.grid_dist_2d(sy, hy, "manhattan", k)
    cx = ((DX * DX) @ u).astype(dt)
    cy = ((DY * DY) @ v).astype(dt)
    s = dt(2.0 * hx ** k * hy ** k)
    return (cx[:, None] + cy[None, :] - s * Z).astype(dt)


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("L", [1, 2, 5, 9])
def test_image_transform_float64_is_the_kronecker_expansion(k, L):
    """In float64 the image transform equals D-hat x with the dense D-hat of
    side L (eq. "2D kronecker"), for every image in a batch."""
    rng = np.random.default_rng(10 * k + L)
    Y = rng.uniform(0.0, 1.0, size=(3, L, L))
    D = O.grid_dist_2d(L, 1.0, "manhattan", k)
    want = (Y.reshape(3, L * L) @ D).reshape(3, L, L)
    got = image_transform(Y, k, np.float64)
    assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("k", [2, 3])
def test_model_float64_matches_oracle(k):
    sx, sy = 4, 5
    rng = np.random.default_rng(k)
    u, v = I.abs_normal_image(sx, rng), I.abs_normal_image(sy, rng)
    T = I.random_coupling(u, v, rng)
    hx, hy = 1 / (sx - 1), 1 / (sy - 1)
    G = model_grad(T, sx, sy, hx, hy, k, u, v, np.float64)
    Gs = O.grad(O.grid_dist_2d(sx, hx, "manhattan", k), O.grid_dist_2d(sy, hy, "manhattan", k), T, u, v)
    assert np.max(np.abs(G - Gs)) <= 1e-13 * np.max(np.abs(Gs))


@pytest.mark.parametrize("k", [2, 3])
def test_model_float32_within_gradient_bound(k):
    """Plain float32 recursions (no compensation) keep the gradient within
    1e-6 relative on 24 x 24 against 32 x 32 grids (n = 576, m = 1024) with
    |N(0,1)| image marginals and the random coupling."""
    sx, sy = 24, 32
    rng = I.rng_for(40 + k)
    u, v = I.abs_normal_image(sx, rng), I.abs_normal_image(sy, rng)
    T = I.random_coupling(u, v, rng).astype(np.float32)
    hx, hy = 1 / (sx - 1), 1 / (sy - 1)
    G = model_grad(T, sx, sy, hx, hy, k, u, v, np.float32)
    Gs = O.grad(O.grid_dist_2d(sx, hx, "manhattan", k), O.grid_dist_2d(sy, hy, "manhattan", k),
                T.astype(np.float64), u, v)
    err = float(np.max(np.abs(G.astype(np.float64) - Gs)) / np.max(np.abs(Gs)))
    assert err <= 1e-6, err

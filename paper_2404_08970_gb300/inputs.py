"""Seeded synthetic inputs for the entropic Gromov-Wasserstein workloads.

This module only draws numbers: marginals on uniform grids, a random positive
coupling with prescribed marginals, image-like 2D intensities and feature
vectors.  It holds none of the method's arithmetic (no distance matrices, no
gradient, no Sinkhorn), so both the CUDA path and the CPU oracle can take their
inputs from here without sharing any computation.

Shapes follow the paper's random-distribution experiments (Sec. 4.1, 1D grids
with random weights; Sec. 4.2, 2D grids on the unit square) and the workload
table used by the benchmark: n = m in {200, 1024, 4096, 8192} for 1D, 64x64
against 96x96 pixels for 2D.
"""
from __future__ import annotations

import numpy as np


def rng_for(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def dirichlet(n: int, alpha: float, rng: np.random.Generator) -> np.ndarray:
    """A Dirichlet(alpha) probability vector of length n, in float64.

    Drawn as normalised Gamma(alpha) variates.  An exact zero (possible for
    small alpha) is redrawn so that every weight is strictly positive and its
    logarithm finite.
    """
    w = rng.gamma(alpha, 1.0, size=n)
    while np.any(w == 0.0):
        z = w == 0.0
        w[z] = rng.gamma(alpha, 1.0, size=int(z.sum()))
    return w / w.sum()


def uniform_weights(n: int) -> np.ndarray:
    return np.full(n, 1.0 / n)


def uniform01_weights(n: int, rng: np.random.Generator) -> np.ndarray:
    """Weights drawn from U[0,1] and normalised (the paper's Sec. 4.1 recipe)."""
    w = rng.uniform(0.0, 1.0, size=n)
    while np.any(w == 0.0):
        z = w == 0.0
        w[z] = rng.uniform(0.0, 1.0, size=int(z.sum()))
    return w / w.sum()


def abs_normal_image(side: int, rng: np.random.Generator) -> np.ndarray:
    """Normalised |N(0,1)| pixel intensities of a side x side image, row-major."""
    w = np.abs(rng.standard_normal(side * side))
    while np.any(w == 0.0):
        z = w == 0.0
        w[z] = np.abs(rng.standard_normal(int(z.sum())))
    return w / w.sum()


def abs_normal_volume(side: int, rng: np.random.Generator) -> np.ndarray:
    """Normalised |N(0,1)| voxel intensities of a side^3 volume, row-major."""
    w = np.abs(rng.standard_normal(side ** 3))
    while np.any(w == 0.0):
        z = w == 0.0
        w[z] = np.abs(rng.standard_normal(int(z.sum())))
    return w / w.sum()


def random_coupling(u: np.ndarray, v: np.ndarray, rng: np.random.Generator,
                    spread: float = 0.2) -> np.ndarray:
    """A random strictly positive n x m coupling whose marginals are u and v.

    T = u v^T * (1 + spread * W), where W is a uniform random matrix centred
    with the weights v along rows and u along columns, so that
    sum_p v_p W_ip = 0 and sum_i u_i W_ip = 0 hold exactly.  Then T 1 = u and
    T^T 1 = v up to rounding, with no iteration.  |W| <= 4, so spread = 0.2
    keeps every entry within [0.2, 1.8] * u_i v_p.
    """
    n, m = u.size, v.size
    R = rng.uniform(-1.0, 1.0, size=(n, m))
    Rv = R @ v
    uR = u @ R
    uRv = float(u @ Rv)
    W = R - Rv[:, None] - uR[None, :] + uRv
    return np.outer(u, v) * (1.0 + spread * W)


def random_positive(n: int, m: int, rng: np.random.Generator) -> np.ndarray:
    """An n x m matrix with entries U(0.5, 1.5) (not a coupling)."""
    return rng.uniform(0.5, 1.5, size=(n, m))


def features(count: int, dim: int, rng: np.random.Generator) -> np.ndarray:
    """count feature vectors of length dim with N(0,1) entries, row-major."""
    return rng.standard_normal((count, dim))


# --------------------------------------------------------------------------
# Named workloads.  Grid spacing h = 1/n for 1D (points x_i = i/n) and
# h = 1/(side-1) for 2D and 3D (the unit square and cube).
# --------------------------------------------------------------------------

def workload_1d_small(seed: int = 0):
    """1D n = m = 200, k = 1, Dirichlet(1) marginals, eps = 1e-2, 20 x 100."""
    rng = rng_for(seed)
    n = m = 200
    u = dirichlet(n, 1.0, rng)
    v = dirichlet(m, 1.0, rng)
    return dict(dim=1, nx=n, ny=m, hx=1.0 / n, hy=1.0 / m, k=1, eps=1e-2,
                n_outer=20, n_inner=100, u=u, v=v)


def workload_1d_grad(n: int, k: int, marginals: str = "uniform", seed: int = 0):
    """1D n x n gradient workload: marginals uniform or Dirichlet(0.5) and a
    random positive coupling with those marginals."""
    rng = rng_for(seed)
    if marginals == "uniform":
        u = uniform_weights(n)
        v = uniform_weights(n)
    elif marginals == "dirichlet":
        u = dirichlet(n, 0.5, rng)
        v = dirichlet(n, 0.5, rng)
    else:
        raise ValueError(marginals)
    T = random_coupling(u, v, rng)
    return dict(dim=1, nx=n, ny=n, hx=1.0 / n, hy=1.0 / n, k=k, eps=1e-2,
                n_outer=20, n_inner=100, u=u, v=v, T=T)


def workload_2d(side_x: int = 64, side_y: int = 96, cost: str = "sqeuclid",
                seed: int = 0):
    """2D side_x^2 x side_y^2 workload on the unit square with |N(0,1)| image
    marginals, eps = 5e-3."""
    rng = rng_for(seed)
    u = abs_normal_image(side_x, rng)
    v = abs_normal_image(side_y, rng)
    return dict(dim=2, nx=side_x, ny=side_y, hx=1.0 / (side_x - 1),
                hy=1.0 / (side_y - 1), k=1, cost=cost, eps=5e-3,
                n_outer=20, n_inner=100, u=u, v=v)


def workload_3d(side_x: int = 16, side_y: int = 21, cost: str = "sqeuclid",
                seed: int = 0):
    """3D side_x^3 x side_y^3 workload on the unit cube with |N(0,1)| voxel
    marginals, eps = 5e-3 (the 2D workload's recipe with a third axis; 16^3
    vs 21^3 has about the point counts of the 64^2 vs 96^2 images)."""
    rng = rng_for(seed)
    u = abs_normal_volume(side_x, rng)
    v = abs_normal_volume(side_y, rng)
    return dict(dim=3, nx=side_x, ny=side_y, hx=1.0 / (side_x - 1),
                hy=1.0 / (side_y - 1), k=1, cost=cost, eps=5e-3,
                n_outer=20, n_inner=100, u=u, v=v)


def workload_batch(count: int = 256, seed: int = 0, lo: int = 256, hi: int = 8192,
                   n_outer: int = 20, n_inner: int = 100):
    """`count` independent 1D problems: n and m drawn independently as
    round(exp(U(ln lo, ln hi))), k uniform in {1, 2}, uniform marginals,
    h = 1/n and 1/m, eps = 1e-2."""
    rng = rng_for(seed)
    out = []
    for _ in range(count):
        n = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        m = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        k = int(rng.integers(1, 3))
        out.append(dict(dim=1, nx=n, ny=m, hx=1.0 / n, hy=1.0 / m, k=k, eps=1e-2, n_outer=n_outer,
                        n_inner=n_inner, u=uniform_weights(n), v=uniform_weights(m)))
    return out


SERVE_KINDS = ("1d", "1d_fgw", "2d", "2d_fgw")


def workload_serve(count: int, rate: float, seed: int = 0, lo: int = 128, hi: int = 16384,
                   n_outer: int = 10, n_inner: int = 50, feat_dim: int = 16):
    """A stream of `count` requests with Poisson arrivals at `rate` per second:
    each of the kinds 1D GW, 1D fused GW, 2D GW, 2D fused GW with probability
    1/4; the point count of each space N log-uniform in [lo, hi] (2D: side
    round(sqrt(N)), squared Euclidean on the unit square, |N(0,1)| image
    marginals; 1D: k = 1, h = 1/N, uniform marginals); fused GW with
    theta = 0.5 and feat_dim-dimensional N(0,1) features; eps = 1e-2."""
    rng = rng_for(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += rng.exponential(1.0 / rate)
        kind = SERVE_KINDS[int(rng.integers(0, 4))]
        nx = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        ny = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        r = dict(arrival=t, kind=kind, eps=1e-2, n_outer=n_outer, n_inner=n_inner, k=1, theta=1.0)
        if kind.startswith("2d"):
            sx, sy = int(round(np.sqrt(nx))), int(round(np.sqrt(ny)))
            r.update(dim=2, nx=sx, ny=sy, hx=1.0 / (sx - 1), hy=1.0 / (sy - 1), cost="sqeuclid",
                     u=abs_normal_image(sx, rng), v=abs_normal_image(sy, rng))
            n, m = sx * sx, sy * sy
        else:
            r.update(dim=1, nx=nx, ny=ny, hx=1.0 / nx, hy=1.0 / ny, cost="pow",
                     u=uniform_weights(nx), v=uniform_weights(ny))
            n, m = nx, ny
        if kind.endswith("fgw"):
            r.update(theta=0.5, phi=features(n, feat_dim, rng), psi=features(m, feat_dim, rng))
        out.append(r)
    return out

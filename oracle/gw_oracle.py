"""Plain FP64 CPU oracle for entropic Gromov-Wasserstein on uniform grids.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import this module.  The CUDA library never
calls it and shares no code with it.

Everything here is the textbook definition written out in float64, slow and
direct, each function citing the part of the paper it follows:

* distance matrices on uniform 1D grids (Sec. 2, eq. "1d distance matrices"),
  2D grids (Sec. 3.1, eq. "2d Dx"; squared-Euclidean added for the 2D
  workload) and 3D grids (the same construction with a third axis),
* the gradient decomposition grad E = C1 - 4 D_X Gamma D_Y (Sec. 2.1); this
  module returns G = grad E / 2 = c_x 1^T + 1 c_y^T - 2 D_X T D_Y,
* the brute-force gradient entry (Sec. 2.1, eq. "gradient entry"),
* the objective E (Sec. 2) and entropy H (eq. "entropic GW"),
* log-domain Sinkhorn for the entropic OT subproblem (Sec. 2.1, eq. "GW
  sinkhorn"; the paper only cites Sinkhorn, the log-domain form with f then g
  updates and a fixed iteration count is this module's reading),
* mirror descent (eqs. "GW proximal gradient" and "GW sinkhorn") with the
  proximal weight tau = eps of the Remark or any tau > 0, optionally with
  warm-started Sinkhorn solves, including the fused-GW cost (Remark "FGW"),
* the paper's O(N) recursion for y = L x (Sec. 3, eqs. "1d y" and "1d
  recursive relation"), kept here as an independently pinned statement of
  the method's core step,
* entropic unbalanced GW (Remark "Entropic algorithm for UGW"): its
  objective, the step cost (1/2) grad E plus the scalar g, log-domain
  unbalanced Sinkhorn with KL-relaxed marginals, and the alternate
  minimisation with mass rescaling,
* the fixed-support GW barycenter (named in the conclusion): entropic GW
  solves against each input and the square-loss update of the barycenter's
  distance matrix.

Parity pins for every function live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------
# Distance matrices
# ---------------------------------------------------------------------------


def grid_dist_1d(n: int, h: float, k: int) -> np.ndarray:
    """d_ij = h^k |i-j|^k on an n-point uniform grid (Sec. 2, eq. "1d distance
    matrices")."""
    idx = np.arange(n, dtype=np.float64)
    return (h ** k) * np.abs(idx[:, None] - idx[None, :]) ** k


def grid_dist_2d(side: int, h: float, cost: str, k: int = 1) -> np.ndarray:
    """Distance matrix of a side x side uniform grid, points flattened
    row-major (index a*side + b).

    cost = "manhattan": h^k (|a-a'| + |b-b'|)^k  (Sec. 3.1, eq. "2d Dx", whose
        block matrix D-hat is the Manhattan distance raised to k).
    cost = "sqeuclid":  h^2 ((a-a')^2 + (b-b')^2)  (squared Euclidean).
    """
    a = np.repeat(np.arange(side, dtype=np.float64), side)
    b = np.tile(np.arange(side, dtype=np.float64), side)
    da = np.abs(a[:, None] - a[None, :])
    db = np.abs(b[:, None] - b[None, :])
    if cost == "manhattan":
        return (h ** k) * (da + db) ** k
    if cost == "sqeuclid":
        return (h ** 2) * (da ** 2 + db ** 2)
    raise ValueError(cost)


def grid_dist_3d(side: int, h: float, cost: str, k: int = 1) -> np.ndarray:
    """Distance matrix of a side x side x side uniform grid, points flattened
    row-major (index (a*side + b)*side + c); the 3D case of the grids of
    Sec. 3.1 ("no essential difference" from 2D).

    cost = "manhattan": h^k (|a-a'| + |b-b'| + |c-c'|)^k.
    cost = "sqeuclid":  h^2 ((a-a')^2 + (b-b')^2 + (c-c')^2).
    """
    idx = np.arange(side ** 3)
    a = (idx // (side * side)).astype(np.float64)
    b = ((idx // side) % side).astype(np.float64)
    c = (idx % side).astype(np.float64)
    da = np.abs(a[:, None] - a[None, :])
    db = np.abs(b[:, None] - b[None, :])
    dc = np.abs(c[:, None] - c[None, :])
    if cost == "manhattan":
        return (h ** k) * (da + db + dc) ** k
    if cost == "sqeuclid":
        return (h ** 2) * (da ** 2 + db ** 2 + dc ** 2)
    raise ValueError(cost)


def grid_dist_3d_rows(side: int, h: float, cost: str, rows, k: int = 1) -> np.ndarray:
    """Rows `rows` of grid_dist_3d(side, h, cost, k), formed without the whole
    matrix (the same definition, for grids too large to hold D in full)."""
    idx = np.arange(side ** 3)
    co = np.stack([idx // (side * side), (idx // side) % side, idx % side], axis=1).astype(np.float64)
    d = np.abs(co[np.asarray(rows)][:, None, :] - co[None, :, :])
    if cost == "manhattan":
        return (h ** k) * d.sum(axis=-1) ** k
    if cost == "sqeuclid":
        return (h ** 2) * (d * d).sum(axis=-1)
    raise ValueError(cost)


# ---------------------------------------------------------------------------
# Gradient
# ---------------------------------------------------------------------------


def grad(DX: np.ndarray, DY: np.ndarray, T: np.ndarray, r: np.ndarray,
         c: np.ndarray) -> np.ndarray:
    """G = (D_X o D_X) r 1^T + 1 ((D_Y o D_Y) c)^T - 2 D_X T D_Y.

    Sec. 2.1: grad E(Gamma) = C1 - 4 D_X Gamma D_Y with
    C1 = 2((D_X o D_X) u 1^T + 1 ((D_Y o D_Y) v)^T); this returns grad E / 2.
    r and c are the marginals used in the constant term: the targets (u, v)
    as the paper writes it, or T's own marginals (T 1, T^T 1).
    """
    cx = (DX * DX) @ r
    cy = (DY * DY) @ c
    return cx[:, None] + cy[None, :] - 2.0 * (DX @ T @ DY)


def grad_exact(DX: np.ndarray, DY: np.ndarray, T: np.ndarray) -> np.ndarray:
    """grad() with T's own marginals r = T 1, c = T^T 1 (exact for any T)."""
    return grad(DX, DY, T, T.sum(axis=1), T.sum(axis=0))


def grad_brute(DX: np.ndarray, DY: np.ndarray, T: np.ndarray) -> np.ndarray:
    """G_ip = sum_{j,q} (d_ij - d_pq)^2 T_jq, i.e. half of the gradient entry
    formula of Sec. 2.1 (eq. "gradient entry").  O(n^2 m^2): tiny inputs only."""
    n, m = T.shape
    G = np.empty((n, m))
    for i in range(n):
        for p in range(m):
            diff = DX[i, :][:, None] - DY[p, :][None, :]
            G[i, p] = float(np.sum(diff * diff * T))
    return G


def grad_rows(DX_rows: np.ndarray, DY: np.ndarray, T: np.ndarray,
              cx_rows: np.ndarray, cy: np.ndarray) -> np.ndarray:
    """Selected rows of G: G[I,:] = cx[I] 1^T + 1 cy^T - 2 (D_X[I,:] T) D_Y.

    The same definition as grad(), evaluated only for the rows I whose
    distance rows D_X[I,:] are passed; used to check large problems on a
    sample of outputs.
    """
    return cx_rows[:, None] + cy[None, :] - 2.0 * ((DX_rows @ T) @ DY)


def objective(DX: np.ndarray, DY: np.ndarray, T: np.ndarray) -> float:
    """E(T) = sum_{i,j,p,q} (d_ij - d_pq)^2 T_ip T_jq (Sec. 2), brute force."""
    n, m = T.shape
    total = 0.0
    for i in range(n):
        for p in range(m):
            diff = DX[i, :][:, None] - DY[p, :][None, :]
            total += T[i, p] * float(np.sum(diff * diff * T))
    return total


def value(DX: np.ndarray, DY: np.ndarray, T: np.ndarray) -> float:
    """E(T) = <G(T; T's marginals), T>, equal to objective() for any T."""
    return float(np.sum(grad_exact(DX, DY, T) * T))


def entropy(T: np.ndarray) -> float:
    """H(T) = sum T (ln T - 1) (eq. "entropic GW"); 0 ln 0 = 0."""
    pos = T > 0
    return float(np.sum(T[pos] * (np.log(T[pos]) - 1.0)) - np.sum(T[~pos]))


def fgw_feature_cost(phi: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """c_ip^2 = ||phi_i - psi_p||^2, the squared feature distance used as the
    linear FGW cost C o C (Remark "FGW")."""
    diff = phi[:, None, :] - psi[None, :, :]
    return np.sum(diff * diff, axis=2)


# ---------------------------------------------------------------------------
# Log-domain Sinkhorn and mirror descent
# ---------------------------------------------------------------------------


def _lse(a: np.ndarray, axis: int) -> np.ndarray:
    """log sum exp along axis with the usual max shift."""
    mx = np.max(a, axis=axis, keepdims=True)
    mx = np.where(np.isfinite(mx), mx, 0.0)
    return np.squeeze(mx, axis=axis) + np.log(np.sum(np.exp(a - mx), axis=axis))


def sinkhorn_log(Pi: np.ndarray, u: np.ndarray, v: np.ndarray, eps: float,
                 n_iter: int, f0=None, g0=None):
    """Entropic OT min <Pi, T> + eps H(T) over couplings of (u, v), solved in
    the log domain (the subproblem of eq. "GW sinkhorn").

    Potentials start at f = g = 0 (unless given); each iteration updates
      f_i = eps ln u_i - eps LSE_p((g_p - Pi_ip) / eps)
      g_p = eps ln v_p - eps LSE_i((f_i - Pi_ip) / eps)
    in that order, for a fixed number of iterations (no early stop).
    """
    n, m = Pi.shape
    f = np.zeros(n) if f0 is None else np.array(f0, dtype=np.float64)
    g = np.zeros(m) if g0 is None else np.array(g0, dtype=np.float64)
    lu = np.log(u)
    lv = np.log(v)
    for _ in range(n_iter):
        f = eps * lu - eps * _lse((g[None, :] - Pi) / eps, axis=1)
        g = eps * lv - eps * _lse((f[:, None] - Pi) / eps, axis=0)
    return f, g


def plan(Pi: np.ndarray, f: np.ndarray, g: np.ndarray, eps: float) -> np.ndarray:
    """T_ip = exp((f_i + g_p - Pi_ip) / eps)."""
    return np.exp((f[:, None] + g[None, :] - Pi) / eps)


def sinkhorn_scaling(K: np.ndarray, u: np.ndarray, v: np.ndarray,
                     n_iter: int):
    """Textbook Sinkhorn matrix scaling a = u / (K b), b = v / (K^T a),
    starting from b = 1.  An independent second statement of the same
    iteration (used only to cross-check sinkhorn_log where K does not
    underflow)."""
    b = np.ones(K.shape[1])
    a = np.ones(K.shape[0])
    for _ in range(n_iter):
        a = u / (K @ b)
        b = v / (K.T @ a)
    return a, b


def mirror_descent(DX: np.ndarray, DY: np.ndarray, u: np.ndarray,
                   v: np.ndarray, eps: float, n_outer: int, n_inner: int,
                   theta: float = 1.0, CC: np.ndarray | None = None,
                   T0: np.ndarray | None = None, grad_scale: float = 2.0,
                   tau: float | None = None, warm_start: bool = False):
    """Entropic (F)GW by mirror descent (Sec. 2.1, eqs. "GW proximal
    gradient" and "GW sinkhorn"): each outer step solves the entropic OT
    problem
      argmin <Pi, Gamma> + tau H(Gamma),  Pi = grad E(T) + (eps - tau) grad H(T),
    with grad H(T) = ln T, and replaces T by its plan.  grad E is
      grad_scale * G(T; u, v)                      (GW, theta = 1)
      (1 - theta) CC + theta * grad_scale * G      (FGW, Remark "FGW")
    with grad_scale = 2 the paper's grad E = 2 G.  tau = None means tau = eps
    (the Remark's choice; the (eps - tau) term then vanishes).  T starts at
    the product coupling u v^T.  Each Sinkhorn solve starts from f = g = 0,
    or with warm_start from the previous step's potentials.

    Returns (T, f, g) after n_outer steps.
    """
    tau = eps if tau is None else tau
    T = np.outer(u, v) if T0 is None else np.array(T0, dtype=np.float64)
    f = np.zeros(u.size)
    g = np.zeros(v.size)
    for l in range(n_outer):
        Pi = grad_scale * grad(DX, DY, T, u, v)
        if theta != 1.0:
            Pi = (1.0 - theta) * CC + theta * Pi
        if tau != eps:
            Pi = Pi + (eps - tau) * np.log(T)
        if warm_start and l > 0:
            f, g = sinkhorn_log(Pi, u, v, tau, n_inner, f0=f, g0=g)
        else:
            f, g = sinkhorn_log(Pi, u, v, tau, n_inner)
        T = plan(Pi, f, g, tau)
    return T, f, g


def fgw_value(DX, DY, T, theta: float, CC) -> float:
    """(1 - theta) <CC, T> + theta E(T)  (Remark "FGW")."""
    lin = 0.0 if CC is None else float(np.sum(CC * T))
    return (1.0 - theta) * lin + theta * value(DX, DY, T)


# ---------------------------------------------------------------------------
# Fixed-support GW barycenter (named in the conclusion as a GW variant the
# fast gradient accelerates; the iteration is the cited barycenter method's
# block coordinate descent with the square loss)
# ---------------------------------------------------------------------------


def barycenter_update(Ts, Cs, lambdas, p: np.ndarray) -> np.ndarray:
    """The distance matrix of the barycenter for fixed couplings T_s (each
    with first marginal p): the minimiser over C of
      sum_s lambda_s sum_{i,j,k,l} (C_ij - C_s,kl)^2 T_s,ik T_s,jl,
    which is C = sum_s lambda_s T_s C_s T_s^T / ((sum_s lambda_s) p p^T)."""
    B = np.zeros((p.size, p.size))
    for lam, T, C in zip(lambdas, Ts, Cs):
        B = B + lam * (T @ C @ T.T)
    return B / (float(np.sum(lambdas)) * np.outer(p, p))


def barycenter(Cs, ps, lambdas, p: np.ndarray, C0: np.ndarray, eps: float, n_iter: int, n_outer: int,
               n_inner: int):
    """Fixed-support GW barycenter: n_iter rounds of (i) an entropic GW solve
    between the barycenter (C, p) and each input (C_s, p_s) by mirror descent
    (n_outer steps of n_inner Sinkhorn iterations, T^0 = p p_s^T each round)
    and (ii) the update of C for those couplings.  Returns (C, [T_s])."""
    C = np.array(C0, dtype=np.float64)
    Ts = []
    for _ in range(n_iter):
        Ts = [mirror_descent(C, Cs_s, p, ps_s, eps, n_outer, n_inner)[0] for Cs_s, ps_s in zip(Cs, ps)]
        C = barycenter_update(Ts, Cs, lambdas, p)
    return C, Ts


# ---------------------------------------------------------------------------
# The paper's O(N) product y = L x (Sec. 3)
# ---------------------------------------------------------------------------


def lower_toeplitz(n: int, k: int) -> np.ndarray:
    """L with L_ij = (i - j)^k for i > j, 0 otherwise (Sec. 3, D-tilde = L + L^T)."""
    idx = np.arange(n, dtype=np.float64)
    d = idx[:, None] - idx[None, :]
    return np.where(d > 0, d, 0.0) ** k * (d > 0)


def binomial_table(k: int) -> list[list[int]]:
    """C(r-1, s-1) for r, s = 1..k+1 (footnote on the binomial coefficients)."""
    return [[math.comb(r - 1, s - 1) if s <= r else 0 for s in range(1, k + 2)]
            for r in range(1, k + 2)]


def fgc_lower(x, k: int, count_ops: bool = False):
    """y = L x by the paper's recursion (Sec. 3, eqs. "1d y" and "1d recursive
    relation"), written in the paper's notation with 1-based i and r.

    States a_{i,r} = sum_{j<i} (i-j)^{r-1} x_j for r = 1..k+1, a_{1,r} = 0, and
      a_{i+1,r} = x_i + sum_{s=1..r} C(r-1, s-1) a_{i,s};
    then y_i = a_{i,k+1}.  The states are evaluated in the paper's order
    a_{11..N1}, ..., a_{1,k+1..N,k+1}.  Works elementwise on numpy arrays, so
    x may be a vector (N,) or a matrix (N, ...) transformed along axis 0; with
    integer x (dtype object or int64) the result is exact.

    With count_ops=True also returns (multiplications, additions) counted as
    the paper does: a multiplication for every binomial factor other than the
    leading a_{i,1} term, an addition for every '+'.
    """
    x = np.asarray(x)
    N = x.shape[0]
    C = binomial_table(k)
    a = [[None] * (k + 2) for _ in range(N + 2)]  # a[i][r], 1-based
    zero = x[0] * 0
    mults = 0
    adds = 0
    for r in range(1, k + 2):
        a[1][r] = zero
        for i in range(1, N):
            acc = x[i - 1] + a[i][1]
            adds += 1
            for s in range(2, r + 1):
                acc = acc + C[r - 1][s - 1] * a[i][s]
                mults += 1
                adds += 1
            a[i + 1][r] = acc
    y = np.stack([a[i][k + 1] for i in range(1, N + 1)], axis=0)
    if count_ops:
        return y, (mults, adds)
    return y


def fgc_apply(x, k: int):
    """D-tilde x = L x + L^T x, with L^T x computed by the same recursion on
    the reversed sequence (Sec. 3: "L^T x can be computed in a similar way")."""
    x = np.asarray(x)
    return fgc_lower(x, k) + fgc_lower(x[::-1], k)[::-1]


def fgc_grad_1d(T: np.ndarray, hx: float, hy: float, k: int,
                r: np.ndarray, c: np.ndarray) -> np.ndarray:
    """G via the paper's fast route: D_X T D_Y = hx^k hy^k D~ (D~ T^T)^T
    (eq. "Dx"), each D~ applied with fgc_apply.  Slow (Python recursion);
    for moderate sizes and as the CPU statement of the paper's method."""
    n, m = T.shape
    Y = fgc_apply(T, k)                    # D~_X T, transform along i
    Z = fgc_apply(Y.T, k).T                # (D~_X T) D~_Y, transform along p
    DXsq = grid_dist_1d(n, hx, k) ** 2
    DYsq = grid_dist_1d(m, hy, k) ** 2
    return (DXsq @ r)[:, None] + (DYsq @ c)[None, :] - 2.0 * (hx ** k) * (hy ** k) * Z


# ---------------------------------------------------------------------------
# Unbalanced GW (Sec. 2.1, Remark "Entropic algorithm for UGW")
# ---------------------------------------------------------------------------


def kl(a: np.ndarray, b: np.ndarray) -> float:
    """KL(a|b) = sum a ln(a/b) - sum a + sum b for positive measures (0 ln 0 = 0)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    pos = a > 0
    return float(np.sum(a[pos] * np.log(a[pos] / b[pos])) - a.sum() + b.sum())


def kl_tensor(a: np.ndarray, b: np.ndarray) -> float:
    """KL(a (x) a | b (x) b) of the tensor-product measures, written out:
    2 m(a) sum a ln(a/b) - m(a)^2 + m(b)^2."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    pos = a > 0
    return float(2.0 * a.sum() * np.sum(a[pos] * np.log(a[pos] / b[pos])) - a.sum() ** 2 + b.sum() ** 2)


def ugw_value(DX, DY, T, u, v, rho: float, eps: float) -> float:
    """The entropic UGW objective of the Remark:
    E(T) + rho KLx(T 1 | u) + rho KLx(T^T 1 | v) + eps KLx(T | u v^T),
    KLx the KL of tensor products (kl_tensor)."""
    return (value(DX, DY, T) + rho * kl_tensor(T.sum(axis=1), u) + rho * kl_tensor(T.sum(axis=0), v)
            + eps * kl_tensor(T, np.outer(u, v)))


def ugw_cost(DX, DY, Th, u, v, rho: float, eps: float) -> np.ndarray:
    """Cost of one UGW step at the current plan Th: (1/2) grad E(Th) = the
    gradient with Th's own marginals, plus the scalar g(Th) = rho KL(Th 1|u)'
    + ... written as the three KL divergences' first-order terms:
      g = rho sum_j r_j ln(r_j/u_j) + rho sum_q c_q ln(c_q/v_q)
          + eps sum_jq Th_jq ln(Th_jq/(u_j v_q)),
    r = Th 1, c = Th^T 1."""
    r, c = Th.sum(axis=1), Th.sum(axis=0)
    g = (rho * float(np.sum(r * np.log(r / u))) + rho * float(np.sum(c * np.log(c / v)))
         + eps * float(np.sum(Th * np.log(Th / np.outer(u, v)))))
    return grad_exact(DX, DY, Th) + g


def sinkhorn_unbalanced(C: np.ndarray, u: np.ndarray, v: np.ndarray, eps: float, rho: float,
                        n_iter: int):
    """min <C, T> + rho KL(T 1|u) + rho KL(T^T 1|v) + eps KL(T|u v^T) in the log
    domain, from f = g = 0, f then g each iteration:
      f_i = -(rho/(rho+eps)) eps LSE_p((g_p - C_ip)/eps + ln v_p)
      g_p = -(rho/(rho+eps)) eps LSE_i((f_i - C_ip)/eps + ln u_i)
    and the plan T_ip = exp((f_i + g_p - C_ip)/eps) u_i v_p."""
    n, m = C.shape
    f = np.zeros(n)
    g = np.zeros(m)
    kappa = rho / (rho + eps)
    lu, lv = np.log(u), np.log(v)
    for _ in range(n_iter):
        f = -kappa * eps * _lse((g[None, :] - C) / eps + lv[None, :], axis=1)
        g = -kappa * eps * _lse((f[:, None] - C) / eps + lu[:, None], axis=0)
    T = np.exp((f[:, None] + g[None, :] - C) / eps) * np.outer(u, v)
    return T, f, g


def ugw_solve(DX, DY, u, v, eps: float, rho: float, n_outer: int, n_inner: int):
    """Entropic UGW by the alternate minimisation the Remark describes: at the
    current plan Th (mass m = sum Th), solve the unbalanced entropic OT
    problem with cost ugw_cost(Th) and penalties scaled by m, i.e. with cost
    C / m and the fixed eps, rho; then rescale the new plan to mass
    sqrt(m(Th) m(T)) (T <- sqrt(m(Th)/m(T)) T).  T starts at
    u v^T / sqrt(m(u) m(v)).  Returns (T, f, g) of the last step."""
    T = np.outer(u, v) / math.sqrt(u.sum() * v.sum())
    f = np.zeros(u.size)
    g = np.zeros(v.size)
    for _ in range(n_outer):
        mh = float(T.sum())
        C = ugw_cost(DX, DY, T, u, v, rho, eps) / mh
        Tn, f, g = sinkhorn_unbalanced(C, u, v, eps, rho, n_inner)
        T = math.sqrt(mh / float(Tn.sum())) * Tn
    return T, f, g

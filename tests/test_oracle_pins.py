"""Pins for the FP64 oracle against facts the paper and the mathematics fix.

None of these tests touches the GPU.  Each pin is chosen so that a plausible
mistake in the oracle (a dropped term, a wrong sign or index, a transposed
operand, a missing factor 2) makes one of them fail; test_planted_mistakes
checks exactly that for a few such mistakes.
"""
import math
import os

import numpy as np
import pytest

from oracle import gw_oracle as O
from paper_2404_08970_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ---------------------------------------------------------------------------
# Printed matrices (golden fixtures typed from the paper)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k,name", [(1, "L_N5_k1.txt"), (2, "L_N5_k2.txt")])
def test_golden_L(k, name):
    assert np.array_equal(O.lower_toeplitz(5, k), load_golden(name))


def test_golden_D1_and_dtilde():
    D1 = load_golden("D1_n4.txt")
    assert np.array_equal(O.grid_dist_1d(4, 1.0, 1), D1)
    L = O.lower_toeplitz(4, 1)
    assert np.array_equal(L + L.T, D1)  # D-tilde = L + L^T (Sec. 3)


@pytest.mark.parametrize("n,k,name", [(2, 1, "Dhat_n2_k1.txt"), (3, 2, "Dhat_n3_k2.txt")])
def test_golden_Dhat(n, k, name):
    assert np.array_equal(O.grid_dist_2d(n, 1.0, "manhattan", k), load_golden(name))


# ---------------------------------------------------------------------------
# The paper's recursion for y = L x (Sec. 3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("N", [1, 2, 3, 7, 40])
def test_recursion_exact_integers(k, N):
    rng = np.random.default_rng(100 * k + N)
    x = rng.integers(-50, 50, size=N).astype(object)
    L = [[(i - j) ** k if i > j else 0 for j in range(N)] for i in range(N)]
    want = [sum(L[i][j] * x[j] for j in range(N)) for i in range(N)]
    got = O.fgc_lower(x, k)
    assert [int(v) for v in got] == [int(v) for v in want]


def stirling2(k, r):
    return sum((-1) ** (r - j) * math.comb(r, j) * j ** k for j in range(r + 1)) // math.factorial(r)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_recursion_vs_stirling_form(k):
    """Independent derivation: t^k = sum_r S2(k,r) r! C(t,r), and
    sum_{j<i} C(i-j, r) x_j is the r-fold shifted (r+1)-fold prefix sum.
    So L x = sum_r S2(k,r) r! shift_r(S^{r+1} x), in exact integers."""
    N = 33
    rng = np.random.default_rng(k)
    x = rng.integers(0, 1000, size=N).astype(np.int64)
    total = np.zeros(N, dtype=np.int64)
    for r in range(1, k + 1):
        s = x.copy()
        for _ in range(r + 1):
            s = np.cumsum(s)
        shifted = np.zeros(N, dtype=np.int64)
        shifted[r:] = s[:N - r]
        total += stirling2(k, r) * math.factorial(r) * shifted
    assert np.array_equal(O.fgc_lower(x, k).astype(np.int64), total)


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("N", [2, 10, 57])
def test_recursion_operation_counts(k, N):
    """Sec. 3: (N-1) k(k+1)/2 multiplications and (N-1)(k+1)(k+2)/2 additions."""
    _, (mults, adds) = O.fgc_lower(np.ones(N), k, count_ops=True)
    assert mults == (N - 1) * k * (k + 1) // 2
    assert adds == (N - 1) * (k + 1) * (k + 2) // 2


@pytest.mark.parametrize("k", [1, 2, 3])
def test_fast_equals_dense_gradient(k):
    """The paper's claim that FGC reproduces the original gradient: the fast
    route (eq. "Dx" with the recursion) equals the dense decomposition."""
    rng = np.random.default_rng(7 + k)
    n, m = 37, 23
    u = I.dirichlet(n, 1.0, rng)
    v = I.dirichlet(m, 1.0, rng)
    T = I.random_coupling(u, v, rng)
    hx, hy = 1.0 / n, 1.0 / m
    DX, DY = O.grid_dist_1d(n, hx, k), O.grid_dist_1d(m, hy, k)
    G_dense = O.grad(DX, DY, T, u, v)
    G_fast = O.fgc_grad_1d(T, hx, hy, k, u, v)
    assert relerr(G_fast, G_dense) < 1e-13


# ---------------------------------------------------------------------------
# Gradient: brute force, closed forms, invariances
# ---------------------------------------------------------------------------

def _tiny_cases():
    cases = []
    for k in (1, 2, 3):
        cases.append(("1d", k, O.grid_dist_1d(5, 0.3, k), O.grid_dist_1d(4, 0.7, k)))
    cases.append(("2d-man1", 1, O.grid_dist_2d(2, 0.5, "manhattan", 1), O.grid_dist_2d(3, 0.5, "manhattan", 1)))
    cases.append(("2d-man2", 2, O.grid_dist_2d(3, 0.5, "manhattan", 2), O.grid_dist_2d(2, 1.0, "manhattan", 2)))
    cases.append(("2d-sq", 2, O.grid_dist_2d(3, 0.5, "sqeuclid"), O.grid_dist_2d(2, 0.25, "sqeuclid")))
    return cases


@pytest.mark.parametrize("case", _tiny_cases(), ids=lambda c: c[0] + f"-k{c[1]}")
def test_grad_matches_brute_force(case):
    _, _, DX, DY = case
    rng = np.random.default_rng(3)
    T = rng.uniform(0.1, 1.0, size=(DX.shape[0], DY.shape[0]))
    assert relerr(O.grad_exact(DX, DY, T), O.grad_brute(DX, DY, T)) < 1e-13


@pytest.mark.parametrize("case", _tiny_cases()[:4], ids=lambda c: c[0] + f"-k{c[1]}")
def test_value_matches_objective(case):
    _, _, DX, DY = case
    rng = np.random.default_rng(4)
    T = rng.uniform(0.0, 1.0, size=(DX.shape[0], DY.shape[0]))
    T /= T.sum()
    E = O.objective(DX, DY, T)
    assert E >= 0
    assert abs(O.value(DX, DY, T) - E) <= 1e-13 * E


def closed_form_dtilde_ones(N, k):
    """(D-tilde 1)_i = sum_{t=1}^{i-1} t^k + sum_{t=1}^{N-i} t^k (1-based i),
    with Faulhaber's sums for k = 1, 2."""
    i = np.arange(1, N + 1, dtype=np.float64)
    if k == 1:
        return (i - 1) * i / 2 + (N - i) * (N - i + 1) / 2
    if k == 2:
        s = lambda t: t * (t + 1) * (2 * t + 1) / 6
        return s(i - 1) + s(N - i)
    raise ValueError(k)


@pytest.mark.parametrize("k", [1, 2])
def test_product_coupling_closed_form(k):
    """T = u v^T with uniform u, v: D_X T D_Y = (D_X u)(D_Y v)^T in closed form,
    and the constant term c_x = (D_X o D_X) u in closed form (k = 1)."""
    n, m = 31, 19
    hx, hy = 1.0 / n, 1.0 / m
    u, v = np.full(n, 1.0 / n), np.full(m, 1.0 / m)
    DX, DY = O.grid_dist_1d(n, hx, k), O.grid_dist_1d(m, hy, k)
    G = O.grad(DX, DY, np.outer(u, v), u, v)
    a = hx ** k * closed_form_dtilde_ones(n, k) / n
    b = hy ** k * closed_form_dtilde_ones(m, k) / m
    cx = hx ** (2 * k) * closed_form_dtilde_ones(n, 2 * k) / n if 2 * k <= 2 else (DX * DX) @ u
    cy = hy ** (2 * k) * closed_form_dtilde_ones(m, 2 * k) / m if 2 * k <= 2 else (DY * DY) @ v
    want = cx[:, None] + cy[None, :] - 2.0 * np.outer(a, b)
    assert relerr(G, want) < 1e-13


@pytest.mark.parametrize("dim", [1, 2])
def test_reflection_equivariance(dim):
    """Reflecting a uniform grid maps D to J D J = D (Sec. 4.3 invariance), so
    G(J T J') = J G(T) J' exactly."""
    rng = np.random.default_rng(11)
    if dim == 1:
        DX, DY = O.grid_dist_1d(9, 0.1, 1), O.grid_dist_1d(7, 0.2, 1)
    else:
        DX, DY = O.grid_dist_2d(3, 0.5, "manhattan", 1), O.grid_dist_2d(4, 0.3, "sqeuclid")
    n, m = DX.shape[0], DY.shape[0]
    T = rng.uniform(size=(n, m))
    r, c = rng.uniform(size=n), rng.uniform(size=m)
    G = O.grad(DX, DY, T, r, c)
    Gr = O.grad(DX, DY, T[::-1, ::-1], r[::-1], c[::-1])
    assert relerr(Gr[::-1, ::-1], G) < 1e-13
    Gc = O.grad(DX, DY, T[:, ::-1], r, c[::-1])
    assert relerr(Gc[:, ::-1], G) < 1e-13


def test_transpose_and_symmetry():
    rng = np.random.default_rng(12)
    DX, DY = O.grid_dist_1d(8, 0.2, 2), O.grid_dist_1d(6, 0.3, 2)
    T = rng.uniform(size=(8, 6))
    r, c = rng.uniform(size=8), rng.uniform(size=6)
    assert relerr(O.grad(DY, DX, T.T, c, r), O.grad(DX, DY, T, r, c).T) < 1e-13
    D = O.grid_dist_1d(7, 0.1, 1)
    S = rng.uniform(size=(7, 7))
    S = S + S.T
    w = rng.uniform(size=7)
    G = O.grad(D, D, S, w, w)
    assert relerr(G, G.T) < 1e-13


def test_linearity():
    rng = np.random.default_rng(13)
    DX, DY = O.grid_dist_1d(6, 0.2, 1), O.grid_dist_1d(5, 0.3, 1)
    A, B = rng.uniform(size=(6, 5)), rng.uniform(size=(6, 5))
    zx, zy = np.zeros(6), np.zeros(5)
    lhs = O.grad(DX, DY, 2.0 * A - 3.0 * B, zx, zy)
    rhs = 2.0 * O.grad(DX, DY, A, zx, zy) - 3.0 * O.grad(DX, DY, B, zx, zy)
    assert relerr(lhs, rhs) < 1e-13


# ---------------------------------------------------------------------------
# 2D structure (Sec. 3.1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", [1, 2, 3])
def test_kronecker_expansion(k):
    """eq. "2D kronecker": D-hat = sum_r C(k,r) D1^{odot r} (x) D1^{odot k-r}
    with D1^{odot 0} = J (0^0 = 1), and D-hat x = sum_r C(k,r)
    vec(D1^{odot k-r} mat(x) D1^{odot r}) with the row-major vec."""
    n = 4
    D1 = O.grid_dist_1d(n, 1.0, 1)
    pw = lambda e: np.ones((n, n)) if e == 0 else D1 ** e
    Dhat = O.grid_dist_2d(n, 1.0, "manhattan", k)
    K = sum(math.comb(k, r) * np.kron(pw(r), pw(k - r)) for r in range(k + 1))
    assert np.array_equal(K, Dhat)
    x = np.random.default_rng(k).uniform(size=n * n)
    y = sum(math.comb(k, r) * (pw(k - r) @ x.reshape(n, n) @ pw(r)).reshape(-1) for r in range(k + 1))
    # With row-major vec, D1^{odot r} (x) D1^{odot k-r} acts as
    # mat(x) -> D1^{odot r} mat(x) D1^{odot k-r}; summing over r symmetrically
    # gives the same total because C(k,r) = C(k,k-r).
    assert relerr(y, Dhat @ x) < 1e-13


@pytest.mark.parametrize("cost", ["sqeuclid", "manhattan"])
def test_2d_four_marginal_identity(cost):
    """For a separable 2D cost d = phi(da) + phi(db) (squared Euclidean, or
    Manhattan with k = 1), D_X T D_Y[(a,b),(c,d)] =
    Z1[a,c] + Z2[a,d] + Z3[b,c] + Z4[b,d], Zt = Phi_X Mt Phi_Y, where the Mt
    are T's sums over the other two grid axes."""
    sx, sy = 3, 4
    hx, hy = 0.5, 0.25
    DX = O.grid_dist_2d(sx, hx, cost, 1)
    DY = O.grid_dist_2d(sy, hy, cost, 1)
    kk = 2 if cost == "sqeuclid" else 1
    PX = O.grid_dist_1d(sx, hx, kk)
    PY = O.grid_dist_1d(sy, hy, kk)
    T = np.random.default_rng(5).uniform(size=(sx * sx, sy * sy))
    T4 = T.reshape(sx, sx, sy, sy)  # [a, b, c, d]
    M1 = T4.sum(axis=(1, 3))  # [a, c]
    M2 = T4.sum(axis=(1, 2))  # [a, d]
    M3 = T4.sum(axis=(0, 3))  # [b, c]
    M4 = T4.sum(axis=(0, 2))  # [b, d]
    Z1, Z2, Z3, Z4 = (PX @ M @ PY for M in (M1, M2, M3, M4))
    Z = (Z1[:, None, :, None] + Z2[:, None, None, :] + Z3[None, :, :, None] + Z4[None, :, None, :])
    assert relerr(Z.reshape(sx * sx, sy * sy), DX @ T @ DY) < 1e-13


# ---------------------------------------------------------------------------
# Sinkhorn and mirror descent
# ---------------------------------------------------------------------------

def _small_problem(n=12, m=9, seed=0):
    rng = np.random.default_rng(seed)
    u, v = I.dirichlet(n, 1.0, rng), I.dirichlet(m, 1.0, rng)
    Pi = rng.uniform(0.0, 1.0, size=(n, m))
    return u, v, Pi


def test_sinkhorn_column_marginals_exact_and_rows_converge():
    u, v, Pi = _small_problem()
    f, g = O.sinkhorn_log(Pi, u, v, 0.1, 200)
    T = O.plan(Pi, f, g, 0.1)
    assert np.max(np.abs(T.sum(axis=0) - v)) < 1e-13
    assert np.max(np.abs(T.sum(axis=1) - u)) < 1e-10
    f1, g1 = O.sinkhorn_log(Pi, u, v, 0.1, 1)
    T1 = O.plan(Pi, f1, g1, 0.1)
    assert np.max(np.abs(T1.sum(axis=0) - v)) < 1e-13


def test_sinkhorn_matches_scaling_form():
    """The log-domain iteration and the textbook scaling iteration are the
    same sequence: T = diag(a) K diag(b), K = exp(-Pi/eps), a = exp(f/eps),
    b = exp(g/eps)."""
    u, v, Pi = _small_problem(seed=1)
    eps = 0.2
    f, g = O.sinkhorn_log(Pi, u, v, eps, 37)
    a, b = O.sinkhorn_scaling(np.exp(-Pi / eps), u, v, 37)
    assert relerr(np.exp(f / eps), a) < 1e-12
    assert relerr(np.exp(g / eps), b) < 1e-12


def test_sinkhorn_large_eps_gives_product_coupling():
    u, v, Pi = _small_problem(seed=2)
    f, g = O.sinkhorn_log(Pi, u, v, 1e7, 5)
    assert relerr(O.plan(Pi, f, g, 1e7), np.outer(u, v)) < 1e-6


def test_mirror_descent_reflection():
    """Reversing v's grid reverses the plan's columns (exact symmetry of the
    uniform grid; the paper's reflection invariance, Sec. 4.3)."""
    n, m = 10, 8
    rng = np.random.default_rng(21)
    u, v = I.dirichlet(n, 1.0, rng), I.dirichlet(m, 1.0, rng)
    DX, DY = O.grid_dist_1d(n, 1.0 / n, 1), O.grid_dist_1d(m, 1.0 / m, 1)
    T, _, _ = O.mirror_descent(DX, DY, u, v, 0.05, 5, 30)
    Tr, _, _ = O.mirror_descent(DX, DY, u, v[::-1].copy(), 0.05, 5, 30)
    assert relerr(Tr[:, ::-1], T) < 1e-11


def test_mirror_descent_single_point():
    """n = 1: the only coupling is T = v^T."""
    rng = np.random.default_rng(22)
    v = I.dirichlet(6, 1.0, rng)
    DX, DY = O.grid_dist_1d(1, 1.0, 1), O.grid_dist_1d(6, 1.0 / 6, 1)
    T, _, _ = O.mirror_descent(DX, DY, np.ones(1), v, 0.05, 3, 10)
    assert relerr(T[0], v) < 1e-13


def test_fgw_limits():
    n, m = 7, 6
    rng = np.random.default_rng(23)
    u, v = I.dirichlet(n, 1.0, rng), I.dirichlet(m, 1.0, rng)
    DX, DY = O.grid_dist_1d(n, 1.0 / n, 1), O.grid_dist_1d(m, 1.0 / m, 1)
    CC = O.fgw_feature_cost(I.features(n, 4, rng), I.features(m, 4, rng))
    Tg, _, _ = O.mirror_descent(DX, DY, u, v, 0.1, 3, 20)
    T1, _, _ = O.mirror_descent(DX, DY, u, v, 0.1, 3, 20, theta=1.0, CC=CC)
    assert relerr(T1, Tg) < 1e-14
    T0, _, _ = O.mirror_descent(DX, DY, u, v, 0.1, 3, 20, theta=0.0, CC=CC)
    f, g = O.sinkhorn_log(CC, u, v, 0.1, 20)
    assert relerr(T0, O.plan(CC, f, g, 0.1)) < 1e-13


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.0])
def test_fgw_value_matches_brute_force(theta):
    """Fused GW objective (Remark "FGW"): (1 - theta) sum_ip c_ip^2 T_ip +
    theta sum_ijpq (D_ij - D'_pq)^2 T_ip T_jq, summed term by term."""
    rng = np.random.default_rng(26)
    n, m = 4, 3
    DX, DY = O.grid_dist_1d(n, 0.5, 2), O.grid_dist_1d(m, 1.0 / 3, 1)
    phi, psi = I.features(n, 3, rng), I.features(m, 3, rng)
    CC = O.fgw_feature_cost(phi, psi)
    T = rng.uniform(0.1, 1.0, size=(n, m))
    lin = sum(CC[i, p] * T[i, p] for i in range(n) for p in range(m))
    quad = sum((DX[i, j] - DY[p, q]) ** 2 * T[i, p] * T[j, q]
               for i in range(n) for j in range(n) for p in range(m) for q in range(m))
    want = (1.0 - theta) * lin + theta * quad
    assert abs(O.fgw_value(DX, DY, T, theta, CC) - want) <= 1e-13 * abs(want)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_fgc_apply_exact_integers(k):
    """D-tilde x = L x + L^T x (Sec. 3) equals the dense |i-j|^k product exactly
    on integer input."""
    N = 9
    x = np.array([3, -1, 4, 1, -5, 9, 2, -6, 5], dtype=object)
    D = [[abs(i - j) ** k for j in range(N)] for i in range(N)]
    want = [sum(D[i][j] * x[j] for j in range(N)) for i in range(N)]
    assert list(O.fgc_apply(x, k)) == want


def test_feature_cost_definition():
    rng = np.random.default_rng(24)
    phi, psi = I.features(5, 3, rng), I.features(4, 3, rng)
    CC = O.fgw_feature_cost(phi, psi)
    for i in range(5):
        for p in range(4):
            assert abs(CC[i, p] - sum((phi[i, t] - psi[p, t]) ** 2 for t in range(3))) < 1e-13


def test_random_coupling_marginals():
    rng = np.random.default_rng(25)
    u, v = I.dirichlet(50, 0.5, rng), I.dirichlet(40, 0.5, rng)
    T = I.random_coupling(u, v, rng)
    assert np.all(T > 0)
    assert np.max(np.abs(T.sum(axis=1) - u)) < 1e-15
    assert np.max(np.abs(T.sum(axis=0) - v)) < 1e-15


# ---------------------------------------------------------------------------
# Planted mistakes: each must be caught by one of the pins above
# ---------------------------------------------------------------------------

def test_planted_mistakes():
    rng = np.random.default_rng(31)
    DX, DY = O.grid_dist_1d(5, 0.3, 1), O.grid_dist_1d(4, 0.7, 1)
    T = rng.uniform(0.1, 1.0, size=(5, 4))
    brute = O.grad_brute(DX, DY, T)
    r, c = T.sum(axis=1), T.sum(axis=0)
    cx, cy = (DX * DX) @ r, (DY * DY) @ c
    wrong = {
        "factor 4 (the paper's grad E scale)": cx[:, None] + cy[None, :] - 4.0 * DX @ T @ DY,
        "dropped c_y": cx[:, None] - 2.0 * DX @ T @ DY,
        "c_y from the wrong marginal": cx[:, None] + ((DY * DY) @ T[:4, :].sum(axis=1))[None, :] - 2.0 * DX @ T @ DY,
        "sign of the bilinear term": cx[:, None] + cy[None, :] + 2.0 * DX @ T @ DY,
        "D_Y built with exponent k + 1": cx[:, None] + cy[None, :] - 2.0 * DX @ T @ O.grid_dist_1d(4, 0.7, 2),
    }
    for name, G in wrong.items():
        assert relerr(G, brute) > 1e-3, name
    # A recursion with the wrong binomial row fails the exact-integer pin.
    x = np.arange(1, 9).astype(object)
    L2 = [[(i - j) ** 2 if i > j else 0 for j in range(8)] for i in range(8)]
    want = [sum(L2[i][j] * x[j] for j in range(8)) for i in range(8)]
    a1 = [0] * 9
    a2 = [0] * 9
    a3 = [0] * 9
    for i in range(1, 8):  # mistake: a3 update uses C(2,1) = 1 instead of 2
        a1[i + 1] = x[i - 1] + a1[i]
        a2[i + 1] = x[i - 1] + a1[i] + a2[i]
        a3[i + 1] = x[i - 1] + a1[i] + 1 * a2[i] + a3[i]
    assert [int(a3[i]) for i in range(1, 9)] != [int(w) for w in want]


# ---------------------------------------------------------------------------
# Entropy (eq. "entropic GW") and the sampled-row gradient
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,m", [(1, 1), (3, 5), (40, 17)])
def test_entropy_product_coupling_closed_form(n, m):
    """Uniform product coupling T = u v^T, T_ip = 1/(nm):
    H = sum T (ln T - 1) = -ln(nm) - 1."""
    T = np.full((n, m), 1.0 / (n * m))
    assert abs(O.entropy(T) - (-math.log(n * m) - 1.0)) < 1e-13


@pytest.mark.parametrize("n", [1, 4, 9])
def test_entropy_with_exact_zeros(n):
    """A permutation coupling T = I / n has n entries 1/n and n^2 - n exact
    zeros; with 0 ln 0 = 0 the entropy is ln(1/n) - 1, finite."""
    T = np.eye(n) / n
    H = O.entropy(T)
    assert math.isfinite(H)
    assert abs(H - (-math.log(n) - 1.0)) < 1e-13


def test_entropy_sinkhorn_identity():
    """For a plan T = exp((f_i + g_p - Pi_ip) / eps), ln T is known exactly, so
    eps H(T) = sum T (f_i + g_p - Pi_ip) - eps sum T.  This fixes the sign and
    the -1 independently of how ln is evaluated."""
    u, v, Pi = _small_problem(seed=7)
    eps = 0.05
    f, g = O.sinkhorn_log(Pi, u, v, eps, 25)
    T = O.plan(Pi, f, g, eps)
    want = float(np.sum(T * (f[:, None] + g[None, :] - Pi))) - eps * float(np.sum(T))
    assert abs(eps * O.entropy(T) - want) <= 1e-13 * abs(want)


def test_entropy_scaling_law():
    """H(cT) = c H(T) + c ln(c) sum T for c > 0 (ln(cT) = ln c + ln T)."""
    rng = np.random.default_rng(41)
    T = rng.uniform(0.0, 1.0, size=(6, 7))
    T[1, 2] = 0.0
    c = 3.7
    want = c * O.entropy(T) + c * math.log(c) * float(np.sum(T))
    assert abs(O.entropy(c * T) - want) <= 1e-13 * abs(want)


def _grad_rows_cases():
    rng = np.random.default_rng(43)
    n, m = 11, 11          # square, so a transposed T would still multiply
    DX, DY = O.grid_dist_1d(n, 0.3, 2), O.grid_dist_1d(m, 0.2, 1)
    T = rng.uniform(0.1, 1.0, size=(n, m))
    yield DX, DY, T, T.sum(axis=1), T.sum(axis=0), [0, 3, 10]
    sx, sy = 3, 4
    DX2 = O.grid_dist_2d(sx, 0.5, "manhattan")
    DY2 = O.grid_dist_2d(sy, 1.0 / 3, "sqeuclid")
    T2 = rng.uniform(0.1, 1.0, size=(sx * sx, sy * sy))
    u2, v2 = I.dirichlet(sx * sx, 1.0, rng), I.dirichlet(sy * sy, 1.0, rng)
    yield DX2, DY2, T2, u2, v2, [8, 1, 4]


def test_grad_rows_equals_selected_rows_of_grad():
    """grad_rows on the rows I (their distance rows and constant terms) is
    exactly the rows I of the full gradient, 1D and 2D."""
    for DX, DY, T, r, c, rows in _grad_rows_cases():
        G = O.grad(DX, DY, T, r, c)
        cx = (DX * DX) @ r
        cy = (DY * DY) @ c
        Gr = O.grad_rows(DX[rows], DY, T, cx[rows], cy)
        assert relerr(Gr, G[rows]) < 1e-14
        # ... and, with T's marginals, equal to the brute-force entry formula.
        if r is not None and np.allclose(r, T.sum(axis=1)):
            assert relerr(Gr, O.grad_brute(DX, DY, T)[rows]) < 1e-12


def test_entropy_and_grad_rows_planted_mistakes():
    """Each plausible mistake in entropy() or grad_rows() fails a pin above."""
    n, m = 3, 5
    T = np.full((n, m), 1.0 / (n * m))
    closed = -math.log(n * m) - 1.0
    no_minus_one = float(np.sum(T * np.log(T)))
    flipped = -O.entropy(T)
    assert abs(no_minus_one - closed) > 0.5 and abs(flipped - closed) > 0.5
    Z = np.eye(4) / 4
    with np.errstate(divide="ignore", invalid="ignore"):
        nan_zero = float(np.sum(Z * (np.log(Z) - 1.0)))
    assert not math.isfinite(nan_zero)
    for DX, DY, T, r, c, rows in _grad_rows_cases():
        G = O.grad(DX, DY, T, r, c)
        cx, cy = (DX * DX) @ r, (DY * DY) @ c
        wrong = {
            "T transposed": cx[rows][:, None] + cy[None, :] - 2.0 * ((DX[rows] @ T.T) @ DY) if T.shape[0] == T.shape[1] else None,
            "constant terms of other rows": cx[rows[::-1]][:, None] + cy[None, :] - 2.0 * ((DX[rows] @ T) @ DY),
            "factor 4": cx[rows][:, None] + cy[None, :] - 4.0 * ((DX[rows] @ T) @ DY),
            "distance rows off by one": cx[rows][:, None] + cy[None, :] - 2.0 * ((DX[np.array(rows) - 1] @ T) @ DY),
        }
        for name, Gr in wrong.items():
            if Gr is not None:
                assert relerr(Gr, G[rows]) > 1e-3, name


# ---------------------------------------------------------------------------
# Mirror descent with tau != eps (eqs. "GW proximal gradient", "GW sinkhorn")
# and warm-started Sinkhorn
# ---------------------------------------------------------------------------

def test_warm_sinkhorn_equals_cold_on_shifted_cost():
    """Starting the log-domain iteration from (f0, g0) is the cold iteration on
    the cost Pi - f0_i - g0_p: every iterate is shifted by (f0, g0) and every
    plan is the same (exact up to rounding)."""
    u, v, Pi = _small_problem(seed=11)
    rng = np.random.default_rng(12)
    f0, g0 = rng.normal(size=u.size) * 0.3, rng.normal(size=v.size) * 0.3
    eps = 0.07
    for it in (1, 3, 17):
        fw, gw = O.sinkhorn_log(Pi, u, v, eps, it, f0=f0, g0=g0)
        Ps = Pi - f0[:, None] - g0[None, :]
        fc, gc = O.sinkhorn_log(Ps, u, v, eps, it)
        assert relerr(O.plan(Pi, fw, gw, eps), O.plan(Ps, fc, gc, eps)) < 1e-12
        assert relerr(fw - f0, fc) < 1e-11 and relerr(gw - g0, gc) < 1e-11


def _md_problem(n=9, m=7, seed=51):
    rng = np.random.default_rng(seed)
    u, v = I.dirichlet(n, 1.0, rng), I.dirichlet(m, 1.0, rng)
    return u, v, O.grid_dist_1d(n, 1.0 / n, 1), O.grid_dist_1d(m, 1.0 / m, 1)


def test_tau_equal_eps_is_the_remark():
    u, v, DX, DY = _md_problem()
    T1, f1, g1 = O.mirror_descent(DX, DY, u, v, 0.05, 4, 30)
    T2, f2, g2 = O.mirror_descent(DX, DY, u, v, 0.05, 4, 30, tau=0.05)
    assert np.array_equal(T1, T2)


def test_tau_first_step_is_entropic_ot_at_tau():
    """From T0 = u v^T, ln T0 = ln u_i + ln v_p is separable, so with the
    Sinkhorn solve converged the first step's plan is the entropic OT plan of
    the cost grad E(T0) at regularisation tau, whatever eps is."""
    u, v, DX, DY = _md_problem()
    eps, tau = 0.08, 0.03
    T1, _, _ = O.mirror_descent(DX, DY, u, v, eps, 1, 3000, tau=tau)
    Pi = 2.0 * O.grad(DX, DY, np.outer(u, v), u, v)
    f, g = O.sinkhorn_log(Pi, u, v, tau, 3000)
    assert relerr(T1, O.plan(Pi, f, g, tau)) < 1e-9


def test_tau_keeps_the_fixed_point():
    """A fixed point of the step satisfies grad E(T) + eps ln T = f + g for any
    tau (the (eps - tau) ln T term and the tau H term combine), so long runs
    with tau = eps and tau = 2 eps reach the same plan, and that plan
    satisfies the fixed-point equation; a sign error in the (eps - tau) term
    moves the fixed point."""
    u, v, DX, DY = _md_problem(7, 6, 52)
    eps, tau = 0.2, 0.4
    Ta, _, _ = O.mirror_descent(DX, DY, u, v, eps, 150, 300)
    Tb, fb, gb = O.mirror_descent(DX, DY, u, v, eps, 300, 300, tau=tau)
    assert relerr(Tb, Ta) < 1e-10
    Pi = 2.0 * O.grad(DX, DY, Tb, u, v)
    assert np.max(np.abs(Pi + eps * np.log(Tb) - fb[:, None] - gb[None, :])) < 1e-10
    # Planted mistake: (tau - eps) instead of (eps - tau).
    T = np.outer(u, v)
    for _ in range(300):
        Pi = 2.0 * O.grad(DX, DY, T, u, v) + (tau - eps) * np.log(T)
        f, g = O.sinkhorn_log(Pi, u, v, tau, 300)
        T = O.plan(Pi, f, g, tau)
    assert relerr(T, Ta) > 1e-4


def test_warm_start_converged_inner_loop_matches_cold():
    """With each Sinkhorn solve converged, warm and cold starts give the same
    mirror-descent iterates."""
    u, v, DX, DY = _md_problem(8, 8, 53)
    Tc, _, _ = O.mirror_descent(DX, DY, u, v, 0.1, 5, 2000)
    Tw, _, _ = O.mirror_descent(DX, DY, u, v, 0.1, 5, 2000, warm_start=True)
    assert relerr(Tw, Tc) < 1e-9


# ---------------------------------------------------------------------------
# Unbalanced GW (Remark "Entropic algorithm for UGW")
# ---------------------------------------------------------------------------

def _ugw_problem(n=9, m=7, seed=3, mass_u=1.3, mass_v=0.8):
    rng = np.random.default_rng(seed)
    u, v = I.dirichlet(n, 1.0, rng) * mass_u, I.dirichlet(m, 1.0, rng) * mass_v
    return u, v, O.grid_dist_1d(n, 1.0 / n, 1), O.grid_dist_1d(m, 1.0 / m, 1)


def test_kl_tensor_is_kl_of_products():
    """KL(a (x) a | b (x) b) summed over all pairs equals the closed form."""
    rng = np.random.default_rng(61)
    a, b = rng.uniform(0.1, 1.0, 5), rng.uniform(0.1, 1.0, 5)
    brute = sum(a[i] * a[j] * math.log(a[i] * a[j] / (b[i] * b[j])) - a[i] * a[j] + b[i] * b[j]
                for i in range(5) for j in range(5))
    assert abs(O.kl_tensor(a, b) - brute) < 1e-13
    assert abs(O.kl(a, b) - sum(a[i] * math.log(a[i] / b[i]) - a[i] + b[i] for i in range(5))) < 1e-14


def test_ugw_value_brute_force():
    """The objective of the Remark summed term by term over (i, j, p, q)."""
    u, v, DX, DY = _ugw_problem(4, 3, 62)
    rng = np.random.default_rng(63)
    T = rng.uniform(0.01, 0.2, size=(4, 3))
    rho, eps = 0.7, 0.05
    r, c = T.sum(axis=1), T.sum(axis=0)
    E = sum((DX[i, j] - DY[p, q]) ** 2 * T[i, p] * T[j, q]
            for i in range(4) for j in range(4) for p in range(3) for q in range(3))
    klx = lambda a, b: sum(a[i] * a[j] * math.log(a[i] * a[j] / (b[i] * b[j])) - a[i] * a[j] + b[i] * b[j]
                           for i in range(len(a)) for j in range(len(a)))
    uv = np.outer(u, v).ravel()
    want = E + rho * klx(r, u) + rho * klx(c, v) + eps * klx(T.ravel(), uv)
    assert abs(O.ugw_value(DX, DY, T, u, v, rho, eps) - want) <= 1e-12 * abs(want)


def test_unbalanced_sinkhorn_kkt():
    """At convergence the relaxed-marginal conditions hold:
    T 1 = u exp(-f / rho) and T^T 1 = v exp(-g / rho)."""
    u, v, _, _ = _ugw_problem(8, 6, 64)
    C = np.random.default_rng(65).uniform(0.0, 1.0, size=(8, 6))
    rho, eps = 0.4, 0.1
    T, f, g = O.sinkhorn_unbalanced(C, u, v, eps, rho, 3000)
    assert relerr(T.sum(axis=1), u * np.exp(-f / rho)) < 1e-10
    assert relerr(T.sum(axis=0), v * np.exp(-g / rho)) < 1e-10


def test_ugw_large_rho_is_balanced_gw():
    """rho -> infinity with unit-mass marginals: the marginal penalties become
    constraints and each step is the balanced entropic step with cost
    (1/2) grad E (mirror descent with grad_scale = 1)."""
    u, v, DX, DY = _ugw_problem(mass_u=1.0, mass_v=1.0)
    Tu, _, _ = O.ugw_solve(DX, DY, u, v, 0.05, 1e7, 5, 100)
    Tb, _, _ = O.mirror_descent(DX, DY, u, v, 0.05, 5, 100, grad_scale=1.0)
    assert relerr(Tu, Tb) < 1e-7


def test_ugw_stationarity_and_monotone_objective():
    """The UGW objective decreases step by step, and the limit is a
    stationary point of the objective: with a = T 1, b = T^T 1, m = sum T,
    setting the derivative of E + rho KLx + rho KLx + eps KLx to zero gives
      G(T)_ip + g(T) + m [rho ln(a_i/u_i) + rho ln(b_p/v_p) + eps ln(T_ip/(u_i v_p))] = 0
    with G the gradient with T's marginals and g the scalar of ugw_cost."""
    u, v, DX, DY = _ugw_problem()
    rho, eps = 0.5, 0.05
    vals = []
    T = np.outer(u, v) / math.sqrt(u.sum() * v.sum())
    for _ in range(400):
        vals.append(O.ugw_value(DX, DY, T, u, v, rho, eps))
        mh = float(T.sum())
        Tn, _, _ = O.sinkhorn_unbalanced(O.ugw_cost(DX, DY, T, u, v, rho, eps) / mh, u, v, eps, rho, 500)
        T = math.sqrt(mh / float(Tn.sum())) * Tn
    assert np.all(np.diff(vals) <= 1e-12)
    a, b, m = T.sum(axis=1), T.sum(axis=0), float(T.sum())
    gsc = rho * np.sum(a * np.log(a / u)) + rho * np.sum(b * np.log(b / v)) + eps * np.sum(T * np.log(T / np.outer(u, v)))
    res = (O.grad_exact(DX, DY, T) + gsc
           + m * (rho * np.log(a / u)[:, None] + rho * np.log(b / v)[None, :] + eps * np.log(T / np.outer(u, v))))
    assert np.max(np.abs(res)) < 1e-8
    # The solver's own loop is the same iteration.
    T2, _, _ = O.ugw_solve(DX, DY, u, v, eps, rho, 400, 500)
    assert relerr(T2, T) < 1e-12


def test_ugw_planted_mistakes():
    """A flipped sign of the scalar g or a missing rho/(rho+eps) factor makes
    the objective increase."""
    u, v, DX, DY = _ugw_problem()
    rho, eps = 0.5, 0.05

    def run(gsign, kappa_rho):
        T = np.outer(u, v) / math.sqrt(u.sum() * v.sum())
        vals = [O.ugw_value(DX, DY, T, u, v, rho, eps)]
        for _ in range(15):
            mh = float(T.sum())
            a, b = T.sum(axis=1), T.sum(axis=0)
            g = rho * np.sum(a * np.log(a / u)) + rho * np.sum(b * np.log(b / v)) + eps * np.sum(T * np.log(T / np.outer(u, v)))
            C = (O.grad_exact(DX, DY, T) + gsign * g) / mh
            Tn, _, _ = O.sinkhorn_unbalanced(C, u, v, eps, kappa_rho, 500)
            T = math.sqrt(mh / float(Tn.sum())) * Tn
            vals.append(O.ugw_value(DX, DY, T, u, v, rho, eps))
        return np.max(np.diff(vals))

    assert run(1.0, rho) <= 1e-12
    assert run(-1.0, rho) > 1e-4
    assert run(1.0, 1e12) > 1e-4


def test_ugw_reflection():
    u, v, DX, DY = _ugw_problem(8, 6, 66)
    T, _, _ = O.ugw_solve(DX, DY, u, v, 0.05, 0.5, 5, 50)
    Tr, _, _ = O.ugw_solve(DX, DY, u, v[::-1].copy(), 0.05, 0.5, 5, 50)
    assert relerr(Tr[:, ::-1], T) < 1e-11


# ---------------------------------------------------------------------------
# 3D grids
# ---------------------------------------------------------------------------

def test_grid_dist_3d_entries():
    """Points (0,0,0), (1,1,1), (0,1,1) of a 2 x 2 x 2 grid (indices 0, 7, 3)."""
    D = O.grid_dist_3d(2, 0.5, "manhattan")
    assert D[0, 7] == 1.5 and D[0, 3] == 1.0 and D[3, 7] == 0.5 and D[7, 7] == 0.0
    S = O.grid_dist_3d(3, 2.0, "sqeuclid")
    i, j = (0 * 3 + 1) * 3 + 2, (2 * 3 + 0) * 3 + 0   # (0,1,2) and (2,0,0)
    assert S[i, j] == 4.0 * (4 + 1 + 4)
    D2 = O.grid_dist_3d(3, 1.0, "manhattan", 2)
    assert D2[i, j] == (2 + 1 + 2) ** 2


@pytest.mark.parametrize("cost,k", [("manhattan", 1), ("manhattan", 2), ("sqeuclid", 1)])
def test_grid_dist_3d_rows_are_rows_of_the_matrix(cost, k):
    rows = [0, 7, 31, 124, 63]
    D = O.grid_dist_3d(5, 0.3, cost, k)
    assert np.array_equal(O.grid_dist_3d_rows(5, 0.3, cost, rows, k), D[rows])
    R = O.grid_dist_3d_rows(5, 0.3, cost, rows, k)
    # point 7 = (0, 1, 2) against point 0: coordinate differences 0, 1, 2
    want = 0.3 ** k * 3 ** k if cost == "manhattan" else 0.09 * 5
    assert abs(R[1, 0] - want) < 1e-15
    # planted mistake: rows off by one
    assert not np.array_equal(R, D[[(r + 1) % 125 for r in rows]])


@pytest.mark.parametrize("cost", ["manhattan", "sqeuclid"])
def test_3d_kronecker_sum(cost):
    """Separable 3D cost: D-hat = A (x) J (x) J + J (x) A (x) J + J (x) J (x) A with
    A the 1D |i-j| (Manhattan) or (i-j)^2 (squared Euclidean) matrix."""
    s = 4
    A = O.grid_dist_1d(s, 1.0, 1 if cost == "manhattan" else 2)
    J = np.ones((s, s))
    want = np.kron(np.kron(A, J), J) + np.kron(np.kron(J, A), J) + np.kron(np.kron(J, J), A)
    assert np.array_equal(O.grid_dist_3d(s, 1.0, cost), want)


@pytest.mark.parametrize("cost", ["manhattan", "sqeuclid"])
def test_3d_nine_marginal_identity(cost):
    """The form the 3D GPU path computes: D_X T D_Y = sum over X axes alpha and
    Y axes beta of (A_X M_ab A_Y)[i_alpha, p_beta], M_ab the sums of T over all
    other axes (side x side matrices)."""
    sx, sy = 3, 4
    rng = np.random.default_rng(71)
    T = rng.uniform(0.0, 1.0, size=(sx ** 3, sy ** 3))
    e = 1 if cost == "manhattan" else 2
    AX, AY = O.grid_dist_1d(sx, 1.0, e), O.grid_dist_1d(sy, 1.0, e)
    T6 = T.reshape(sx, sx, sx, sy, sy, sy)
    Z = np.zeros((sx, sx, sx, sy, sy, sy))
    for al in range(3):
        for be in range(3):
            keep = [al, 3 + be]
            M = T6.sum(axis=tuple(q for q in range(6) if q not in keep))   # sx x sy
            Zab = AX @ M @ AY
            shape = [1] * 6
            shape[al], shape[3 + be] = sx, sy
            Z = Z + Zab.reshape(shape)
    want = O.grid_dist_3d(sx, 1.0, cost) @ T @ O.grid_dist_3d(sy, 1.0, cost)
    assert relerr(Z.reshape(sx ** 3, sy ** 3), want) < 1e-13


def test_3d_gradient_matches_brute_force():
    sx, sy = 2, 3
    rng = np.random.default_rng(72)
    T = rng.uniform(0.1, 1.0, size=(sx ** 3, sy ** 3))
    DX, DY = O.grid_dist_3d(sx, 0.7, "sqeuclid"), O.grid_dist_3d(sy, 0.4, "sqeuclid")
    assert relerr(O.grad_exact(DX, DY, T), O.grad_brute(DX, DY, T)) < 1e-12


# ---------------------------------------------------------------------------
# Fixed-support GW barycenter
# ---------------------------------------------------------------------------

def _bary_objective(C, Cs, Ts, lambdas):
    """sum_s lambda_s sum_{i,j,k,l} (C_ij - C_s,kl)^2 T_s,ik T_s,jl, summed term by term."""
    tot = 0.0
    for lam, Csk, T in zip(lambdas, Cs, Ts):
        d = C[:, :, None, None] - Csk[None, None, :, :]          # (i, j, k, l)
        w = T[:, None, :, None] * T[None, :, None, :]           # T_ik T_jl
        tot += lam * float(np.sum(d * d * w))
    return tot


def _bary_case(seed=0):
    rng = np.random.default_rng(seed)
    p = rng.dirichlet(np.ones(4))
    Cs = [O.grid_dist_1d(5, 0.3, 1), O.grid_dist_1d(3, 0.5, 2)]
    ps = [rng.dirichlet(np.ones(5)), rng.dirichlet(np.ones(3))]
    Ts = [I.random_coupling(p, q, rng, spread=0.8) for q in ps]
    return p, Cs, Ts, [0.25, 0.5]


def test_barycenter_update_minimises_the_objective():
    """The update's C is the stationary point (and, the objective being a
    convex quadratic in C, the minimiser) of the brute-force objective for
    fixed couplings: every central difference vanishes, every perturbation
    increases it.  Planted mistakes (weights not normalised, transposed
    couplings) are not stationary."""
    p, Cs, Ts, lam = _bary_case()
    C = O.barycenter_update(Ts, Cs, lam, p)
    f0 = _bary_objective(C, Cs, Ts, lam)
    h = 1e-4
    for i in range(4):
        for j in range(4):
            E = np.zeros((4, 4))
            E[i, j] = h
            dfd = (_bary_objective(C + E, Cs, Ts, lam) - _bary_objective(C - E, Cs, Ts, lam)) / (2 * h)
            assert abs(dfd) < 1e-9, (i, j, dfd)
    rng = np.random.default_rng(3)
    for _ in range(5):
        assert _bary_objective(C + 1e-3 * rng.standard_normal((4, 4)), Cs, Ts, lam) > f0
    B = sum(l * (T @ Ck @ T.T) for l, T, Ck in zip(lam, Ts, Cs))
    unnormalised = B / np.outer(p, p)
    one_sided = B / (float(np.sum(lam)) * p[:, None])
    for bad in (unnormalised, one_sided):
        worst = 0.0
        for i in range(4):
            for j in range(4):
                E = np.zeros((4, 4))
                E[i, j] = h
                d = (_bary_objective(bad + E, Cs, Ts, lam) - _bary_objective(bad - E, Cs, Ts, lam)) / (2 * h)
                worst = max(worst, abs(d))
        assert worst > 1e-6


def test_barycenter_update_identity_coupling_returns_the_input():
    """With the identity coupling T = diag(p) of a space with itself the
    update gives that space's distance matrix back exactly."""
    p = np.array([0.1, 0.2, 0.3, 0.4])
    C1 = O.grid_dist_1d(4, 0.25, 2)
    assert np.allclose(O.barycenter_update([np.diag(p)], [C1], [1.0], p), C1, rtol=0, atol=1e-15)


def test_barycenter_is_symmetric_and_uses_the_solver():
    """The barycenter of symmetric inputs stays symmetric, and its couplings
    are the mirror-descent solves against the final round's barycenter input."""
    rng = np.random.default_rng(5)
    Cs = [O.grid_dist_1d(6, 0.2, 1), O.grid_dist_1d(8, 1 / 8, 2)]
    ps = [rng.dirichlet(np.ones(6)), rng.dirichlet(np.ones(8))]
    p = np.full(5, 0.2)
    C0 = rng.uniform(0, 1, (5, 5))
    C0 = (C0 + C0.T) / 2
    C1, _ = O.barycenter(Cs, ps, [0.3, 0.7], p, C0, 0.05, 1, 3, 30)
    C2, Ts = O.barycenter(Cs, ps, [0.3, 0.7], p, C0, 0.05, 2, 3, 30)
    assert np.max(np.abs(C2 - C2.T)) < 1e-15
    T_direct = O.mirror_descent(C1, Cs[0], p, ps[0], 0.05, 3, 30)[0]
    assert relerr(Ts[0], T_direct) < 1e-14
    assert relerr(O.barycenter_update(Ts, Cs, [0.3, 0.7], p), C2) < 1e-14

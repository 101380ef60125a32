"""Pins for the oracle's per-direction form: one diffusion coefficient per direction
(Sec. 5, Example 4: -sum_j d/dx_j (beta_j d u/dx_j) + alpha u) and separate truncation
degrees per coefficient and per direction (Sec. 4.1's t_1 for beta and t_2 for alpha;
Example 4's t_1j).  Each pin checks the oracle against something other than itself:
the dense quadrature matrix built from its definition, the Kronecker closed form for
constant coefficients, M = K exactly when the coefficients are polynomials within the
stated degrees, the numeric nonzeros of such a matrix for the structural pattern, and a
dense linear solve for PCG.  These run without a GPU.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2004_13961_gb300 import workloads as W


def _grid(d, Q):
    x = W.nodes(Q)
    mesh = np.meshgrid(*([x] * d), indexing="ij")  # mesh[k] varies along axis k (k = 0 slowest)
    # x fastest: direction 0 is the last axis of the C-ordered array
    return [mesh[d - 1 - i].ravel() for i in range(d)]


def _poly1(x, coef):
    return np.polynomial.legendre.legval(x, coef)


def _mass_1d(n1):
    M = np.zeros((n1, n1))
    for k in range(n1):
        M[k, k] = 2.0 / (2 * k + 1) + 2.0 / (2 * k + 5)
        if k + 2 < n1:
            M[k, k + 2] = M[k + 2, k] = -2.0 / (2 * k + 5)
    return M


@pytest.mark.parametrize("d,N", [(1, 9), (2, 7), (2, 6), (3, 5)])
def test_dir_matrix_free_matches_dense_quadrature_matrix(d, N):
    rng = np.random.default_rng(100 + d + N)
    for Q in (N + 1, N + 2):
        nq = Q ** d
        a = [0.5 + rng.random(nq) for _ in range(d)]
        b = rng.random(nq)
        K = O.dense_K_dir(d, N, Q, a, b)
        u = rng.standard_normal((N - 1) ** d)
        y = O.apply_K_dir(d, N, Q, a, b, u)
        assert np.abs(y - K @ u).max() <= 1e-13 * np.abs(K @ u).max()
        assert np.abs(K - K.T).max() <= 1e-13 * np.abs(K).max()


@pytest.mark.parametrize("d,N", [(2, 7), (3, 5)])
def test_dir_constant_coefficients_kronecker_closed_form(d, N):
    """beta_j = c_j, alpha = c: K = sum_j c_j (M x .. S_j .. x M) + c (M x M (x M)) with
    S = diag(4k+6) (Sec. 3) and the pentadiagonal mass matrix."""
    Q, n1 = N + 2, N - 1
    cs, cb = [0.7, 1.9, 3.1][:d], 0.45
    S, M = np.diag(4.0 * np.arange(n1) + 6.0), _mass_1d(n1)

    def kron(mats):  # mats[i] acts on direction i; direction 0 is fastest
        out = np.ones((1, 1))
        for m in reversed(mats):
            out = np.kron(out, m)
        return out

    ref = sum(cs[j] * kron([S if i == j else M for i in range(d)]) for j in range(d))
    ref = ref + cb * kron([M] * d)
    nq = Q ** d
    a = [np.full(nq, c) for c in cs]
    K = O.dense_K_dir(d, N, Q, a, np.full(nq, cb))
    assert np.abs(K - ref).max() < 1e-12 * np.abs(ref).max()
    u = np.random.default_rng(4).standard_normal(n1 ** d)
    assert np.abs(O.apply_K_dir(d, N, Q, a, np.full(nq, cb), u) - ref @ u).max() < 1e-12 * np.abs(ref @ u).max()


def test_dir_truncation_keeps_per_direction_degrees():
    d, Q, T = 2, 12, 5
    rng = np.random.default_rng(6)
    c = rng.standard_normal((T + 1, T + 1))  # c[tx, ty]
    vals = W._grid_eval(d, Q, c).ravel()
    chat = O.coef_trunc_dir(d, Q, T, [3, 1], vals).reshape(T + 1, T + 1)  # [ty, tx]: x degree fastest
    ref = c.copy()
    ref[4:, :] = 0.0  # x degree > 3
    ref[:, 2:] = 0.0  # y degree > 1
    assert np.abs(chat - ref.T).max() < 1e-13


def _example4_like(d, N, Q, degs, tb, has_b, seed):
    """beta_j a polynomial in x_j alone of degree degs[j] (as Example 4's beta_j(x_j)), alpha a
    tensor polynomial of degree tb[i] in direction i, all positive on the square."""
    rng = np.random.default_rng(seed)
    g = _grid(d, Q)
    a = []
    for j in range(d):
        coef = np.zeros(degs[j] + 1)
        coef[0] = 3.0
        coef[1:] = 0.4 * rng.standard_normal(degs[j]) / np.arange(1, degs[j] + 1)
        a.append(_poly1(g[j], coef))
    b = np.ones(Q ** d)
    if has_b:
        for i in range(d):
            coef = np.zeros(tb[i] + 1)
            coef[0] = 1.0
            coef[1:] = 0.2 * rng.standard_normal(tb[i]) / np.arange(1, tb[i] + 1)
            b = b * _poly1(g[i], coef)
    else:
        b = np.zeros(Q ** d)
    return a, b


@pytest.mark.parametrize("d,N,degs,tb,has_b", [
    (2, 9, [4, 2], [2, 1], True),    # Example-4-like, with a reaction term of other degrees
    (2, 8, [5, 3], [0, 0], False),   # Example 4 (a): beta_1(x), beta_2(y), alpha = 0
    (3, 6, [3, 1, 2], [1, 0, 1], True),
])
def test_dir_M_equals_K_for_polynomials_within_degrees(d, N, degs, tb, has_b):
    """With beta_j of degree t_1j in x_j alone and alpha within degrees tb, the truncation drops
    nothing and Q = N + 3 points integrate every product exactly, so the assembled M is K."""
    Q = N + 3
    a, b = _example4_like(d, N, Q, degs, tb, has_b, seed=11 + d)
    ta = [[degs[j] if i == j else 0 for i in range(d)] for j in range(d)]
    st = O.setup_dir(d, N, Q, a, b, ta, tb)
    K = O.dense_K_dir(d, N, Q, a, b)
    assert np.abs(st["M"].to_dense() - K).max() < 1e-13 * np.abs(K).max()


@pytest.mark.parametrize("d,N,ta,tb,has_b", [
    (2, 14, [[4, 0], [0, 3]], [0, 0], False),  # Example 4 (a) degrees t_11 = 4, t_12 = 3
    (2, 12, [[2, 2], [2, 2]], [1, 1], True),   # Sec. 4.1: t_1 = 2 for beta, t_2 = 1 for alpha
    (2, 12, [[3, 1], [0, 2]], [0, 2], True),
    (3, 8, [[2, 0, 0], [0, 1, 0], [0, 0, 3]], [0, 0, 0], True),
])
def test_dir_pattern_is_the_numeric_support(d, N, ta, tb, has_b):
    """The structural pattern equals the set of entries that are nonzero for generic
    coefficients of exactly those degrees: polynomial coefficients, M = K computed by dense
    quadrature, whose nonzeros must be exactly the pattern's positions."""
    Q = N + 6
    rng = np.random.default_rng(21)
    g = _grid(d, Q)

    def tensor_poly(deg, c0):
        v = np.full(Q ** d, 1.0)
        for i in range(d):
            coef = np.zeros(deg[i] + 1)
            coef[0] = c0
            coef[1:] = 0.3 * (0.5 + rng.random(deg[i]))
            v = v * _poly1(g[i], coef)
        return v

    a = [tensor_poly(ta[j], 2.0) for j in range(d)]
    b = tensor_poly(tb, 1.0) if has_b else np.zeros(Q ** d)
    K = O.dense_K_dir(d, N, Q, a, b)
    st = O.setup_dir(d, N, Q, a, b, ta, tb)
    M = st["M"]
    pat = np.zeros_like(K, dtype=bool)
    for r in range(M.n):
        pat[r, M.col[M.rowptr[r]:M.rowptr[r + 1]]] = True
    nz = np.abs(K) > 1e-12 * np.abs(K).max()
    assert np.array_equal(nz, pat)
    assert O.pattern_nnz_dir(d, N, ta, tb, has_b) == pat.sum()
    assert np.abs(M.to_dense() - K).max() < 1e-12 * np.abs(K).max()


def test_dir_isotropic_case_reduces_to_one_coefficient():
    """beta_j all equal, one degree: the per-direction form gives the isotropic oracle's M and
    K x (up to the order of the additions)."""
    d, N, T = 2, 14, 3
    p = W.random_exp_problem(d, N, T, 1, 2, 3)
    st = O.setup(d, N, p["Q"], T, p["a"], p["b"])
    sd = O.setup_dir(d, N, p["Q"], [p["a"]] * d, p["b"], [[T] * d] * d, [T] * d)
    assert np.array_equal(st["M"].col, sd["M"].col)
    assert np.abs(st["M"].val - sd["M"].val).max() < 1e-14 * np.abs(st["M"].val).max()
    u = np.random.default_rng(2).standard_normal((N - 1) ** d)
    y1 = O.apply_K(d, N, p["Q"], p["a"], p["b"], u)
    y2 = O.apply_K_dir(d, N, p["Q"], [p["a"]] * d, p["b"], u)
    assert np.array_equal(y1, y2)


@pytest.mark.parametrize("d,N", [(2, 9), (3, 6)])
def test_dir_pcg_matches_dense_solve(d, N):
    Q = N + 2
    rng = np.random.default_rng(31)
    nq = Q ** d
    a = [np.exp(0.8 * rng.standard_normal() * _grid(d, Q)[j]) for j in range(d)]
    b = np.zeros(nq)
    F = rng.standard_normal((N - 1) ** d)
    ta = [[3 if i == j else 0 for i in range(d)] for j in range(d)]
    r = O.solve_dir(d, N, Q, a, b, ta, [0] * d, F, eps=1e-13)
    assert r["status"] == 0 and r["ilu_status"] == 0
    x = np.linalg.solve(O.dense_K_dir(d, N, Q, a, b), F)
    assert np.abs(r["x"] - x).max() < 1e-11 * np.abs(x).max()


# --------------------------------------------------------------------------- PCG-I (Sec. 5)


@pytest.mark.parametrize("d,N", [(1, 12), (2, 9), (3, 6)])
def test_const_preconditioner_is_the_mean_coefficient_operator(d, N):
    """M_0 (all degrees 0) is the operator with each coefficient replaced by its mean over the
    square (the constant Legendre term): sum_j mean(beta_j) (M x .. S_j .. x M) + mean(alpha) M^d
    with S = diag(4k+6) and the pentadiagonal mass matrix; the means by a plain quadrature sum."""
    Q, n1 = N + 2, N - 1
    rng = np.random.default_rng(40 + d)
    g = _grid(d, Q)
    a = [np.exp(0.5 * np.sin(1.0 + j + g[j]) + 0.2 * g[-1]) for j in range(d)]
    b = 1.0 + 0.3 * np.cos(sum(g))
    x, w = np.polynomial.legendre.leggauss(Q)
    Wt = np.ones(1)
    for _ in range(d):
        Wt = np.kron(w, Wt)
    mean = lambda v: float(Wt @ v) / 2 ** d
    S, M = np.diag(4.0 * np.arange(n1) + 6.0), _mass_1d(n1)

    def kron(mats):
        out = np.ones((1, 1))
        for m in reversed(mats):
            out = np.kron(out, m)
        return out

    ref = sum(mean(a[j]) * kron([S if i == j else M for i in range(d)]) for j in range(d)) + mean(b) * kron([M] * d)
    st = O.setup_const(d, N, Q, a, b)
    assert np.abs(st["dense"] - ref).max() < 1e-13 * np.abs(ref).max()
    assert abs(st["abar"][0] - mean(a[0])) < 1e-14 * abs(mean(a[0]))


def test_const_preconditioner_exact_for_constant_coefficients():
    """Constant coefficients: M_0 = K, so PCG-I converges in one iteration."""
    d, N, Q = 2, 12, 14
    nq = Q ** d
    a, b = [np.full(nq, 1.7), np.full(nq, 0.6)], np.full(nq, 2.5)
    F = np.random.default_rng(2).standard_normal((N - 1) ** d)
    r = O.pcg_const(d, N, Q, a, b, F, eps=1e-12)
    assert r["status"] == 0 and r["iters"] == 1
    assert np.abs(r["setup"]["dense"] - O.dense_K_dir(d, N, Q, a, b)).max() < 1e-12


@pytest.mark.parametrize("d,N", [(2, 10), (3, 6)])
def test_const_pcg_matches_dense_solve(d, N):
    Q = N + 1
    g = _grid(d, Q)
    a = [np.exp(g[j]) for j in range(d)]
    b = np.cos(sum(g))
    F = np.random.default_rng(5).standard_normal((N - 1) ** d)
    r = O.pcg_const(d, N, Q, a, b, F, eps=1e-13)
    assert r["status"] == 0
    x = np.linalg.solve(O.dense_K_dir(d, N, Q, a, b), F)
    assert np.abs(r["x"] - x).max() < 1e-11 * np.abs(x).max()

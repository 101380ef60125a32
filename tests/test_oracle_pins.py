"""Pins for the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: library
routines (numpy's Gauss rule and Legendre series), closed forms that follow from
orthogonality (Sec. 2.1), Lemma 2.1's product linearisation, brute-force dense
matrices, factorisation identities, and the iteration counts the paper prints
(Table 5.7).  These run without a GPU.
"""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle as O
from paper_2004_13961_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def rand_pos(rng, n, lo=0.5):
    return lo + rng.random(n)


# --------------------------------------------------------------------------- Sec. 2


@pytest.mark.parametrize("Q", [1, 2, 3, 7, 10, 33, 130, 514])
def test_gauss_matches_numpy_leggauss(Q):
    x, w = O.gauss(Q)
    xr, wr = npleg.leggauss(Q)
    assert np.all(np.diff(x) > 0)
    assert np.abs(x - xr).max() < 4e-15
    # numpy's endpoint weights lose ~1e-10 relative at large Q (see the mpmath pin below)
    assert np.abs((w - wr) / wr).max() < (1e-13 if Q <= 40 else 1e-9)
    assert np.allclose(x, -x[::-1], atol=0, rtol=0)


def test_gauss_high_precision_large_Q():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    Q = 514
    x, w = O.gauss(Q)
    for i in (0, 1, 7, 100, 256):
        xt = mp.findroot(lambda t: mp.legendre(Q, t), mp.mpf(x[i]))
        wt = 2 / ((1 - xt ** 2) * mp.diff(lambda t: mp.legendre(Q, t), xt) ** 2)
        assert abs(float(x[i] - xt)) < 1e-16
        assert abs(float((w[i] - wt) / wt)) < 1e-11


@pytest.mark.parametrize("Q", [4, 9, 20])
def test_gauss_exact_for_polynomials(Q):
    x, w = O.gauss(Q)
    assert abs(w.sum() - 2.0) < 1e-14
    for p in range(2 * Q):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.dot(w, x ** p) - exact) < 1e-13


def test_legendre_recurrence_vs_numpy_and_endpoints():
    for xv in [-1.0, -0.7, 0.0, 0.3, 1.0]:
        L = O.legendre_all(40, xv)
        ref = [npleg.legval(xv, np.eye(41)[n]) for n in range(41)]
        assert np.abs(L - ref).max() < 1e-13
    L1, Lm1 = O.legendre_all(30, 1.0), O.legendre_all(30, -1.0)
    assert np.allclose(L1, 1.0) and np.allclose(Lm1, [(-1.0) ** n for n in range(31)])


def test_derivative_recurrence_vs_numpy_legder():
    for xv in [-0.9, -0.2, 0.5, 0.95]:
        dL = O.legendre_deriv_all(25, xv)
        ref = [npleg.legval(xv, npleg.legder(np.eye(26)[n])) for n in range(26)]
        assert np.abs(dL - ref).max() < 1e-11
        # phi'_k = -(2k+3) L_{k+1} (derivative recurrence, Sec. 2.1)
        L = O.legendre_all(26, xv)
        for k in range(23):
            assert abs((dL[k] - dL[k + 2]) + (2 * k + 3) * L[k + 1]) < 1e-11


# --------------------------------------------------------------------------- Sec. 3 / 4.3


@pytest.mark.parametrize("d,N", [(1, 9), (2, 7), (2, 6), (3, 5)])
def test_matrix_free_matches_dense_quadrature_matrix(d, N):
    rng = np.random.default_rng(10 + d + N)
    for Q in (N + 1, N + 2):
        nq = Q ** d
        a, b = rand_pos(rng, nq), rng.random(nq)
        K = O.dense_K(d, N, Q, a, b)
        u = rng.standard_normal((N - 1) ** d)
        y = O.apply_K(d, N, Q, a, b, u)
        ref = K @ u
        assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


def _mass_1d(n1):
    M = np.zeros((n1, n1))
    for k in range(n1):
        M[k, k] = 2.0 / (2 * k + 1) + 2.0 / (2 * k + 5)
        if k + 2 < n1:
            M[k, k + 2] = M[k + 2, k] = -2.0 / (2 * k + 5)
    return M


def test_1d_stiffness_is_diagonal():
    N = 11
    Q = N + 2
    K = O.dense_K(1, N, Q, np.ones(Q), np.zeros(Q))
    assert np.abs(K - np.diag(4.0 * np.arange(N - 1) + 6.0)).max() < 1e-12
    u = np.random.default_rng(1).standard_normal(N - 1)
    assert np.abs(O.apply_K(1, N, Q, np.ones(Q), np.zeros(Q), u) - (4 * np.arange(N - 1) + 6) * u).max() < 1e-12


@pytest.mark.parametrize("d,N", [(1, 10), (2, 7), (3, 5)])
def test_constant_coefficient_closed_form(d, N):
    """a=1, b=c: K is the Kronecker sum of diag(4k+6) and the pentadiagonal mass matrix."""
    c = 0.7
    Q = N + 2
    n1 = N - 1
    S, M = np.diag(4.0 * np.arange(n1) + 6.0), _mass_1d(n1)
    if d == 1:
        ref = S + c * M
    elif d == 2:
        ref = np.kron(M, S) + np.kron(S, M) + c * np.kron(M, M)
    else:
        ref = (np.kron(np.kron(M, M), S) + np.kron(np.kron(M, S), M) + np.kron(np.kron(S, M), M)
               + c * np.kron(np.kron(M, M), M))
    nq = Q ** d
    K = O.dense_K(d, N, Q, np.ones(nq), np.full(nq, c))
    assert np.abs(K - ref).max() < 1e-12
    u = np.random.default_rng(2).standard_normal(n1 ** d)
    assert np.abs(O.apply_K(d, N, Q, np.ones(nq), np.full(nq, c), u) - ref @ u).max() < 1e-12


def test_K_symmetric_positive_definite():
    rng = np.random.default_rng(3)
    N, Q = 8, 10
    K = O.dense_K(2, N, Q, rand_pos(rng, Q * Q), rng.random(Q * Q))
    assert np.abs(K - K.T).max() < 1e-12 * np.abs(K).max()
    np.linalg.cholesky(K)


@pytest.mark.parametrize("d,N", [(1, 20), (2, 9), (3, 6)])
def test_load_vector_quadrature_equals_closed_form(d, N):
    Q = N + 2
    st = W.Stream(77 + d)
    fc = W.rhs_coeffs(d, N, st)
    f = W.rhs_samples_from_coeffs(d, Q, fc)
    Fq = O.load_vector(d, N, Q, f)
    Fc = O.load_vector_legendre(d, N, fc.T.copy() if d > 1 else fc)
    assert np.abs(Fq - Fc).max() < 1e-13 * np.abs(Fc).max()


# --------------------------------------------------------------------------- Sec. 4.1 / 4.2


@pytest.mark.parametrize("d", [1, 2, 3])
def test_coefficient_truncation_recovers_polynomial(d):
    T, Q = 4, 9
    rng = np.random.default_rng(4 + d)
    c = rng.standard_normal((T + 1,) * d)
    vals = W._grid_eval(d, Q, c).ravel()
    chat = O.coef_trunc(d, Q, T, vals)
    assert np.abs(chat - c.T.ravel()).max() < 1e-13


def _carlitz_C(r):
    v = 1.0
    for i in range(1, r + 1):
        v *= (2.0 * i - 1.0) / (2.0 * i)
    return v


def _carlitz_inner(t, a, b):
    """(L_t L_a, L_b) from the product linearisation of Lemma 2.1."""
    for s in range(0, min(t, a) + 1):
        if t + a - 2 * s == b:
            coef = ((t + a + 0.5 - 2 * s) / (t + a + 0.5 - s)) * _carlitz_C(s) * _carlitz_C(t - s) \
                * _carlitz_C(a - s) / _carlitz_C(t + a - s)
            return coef * 2.0 / (2 * b + 1)
    return 0.0


def test_band_matrices_match_lemma_2_1():
    N, T = 14, 5
    S, M = O.band_matrices(N, T)
    n1 = N - 1
    for t in range(T + 1):
        for i in range(n1):
            for m in range(n1):
                if abs(i - m) > T + 2:
                    continue
                s_ref = (2 * i + 3) * (2 * m + 3) * _carlitz_inner(t, i + 1, m + 1)
                m_ref = (_carlitz_inner(t, i, m) - _carlitz_inner(t, i, m + 2)
                         - _carlitz_inner(t, i + 2, m) + _carlitz_inner(t, i + 2, m + 2))
                assert abs(S[t, i, m] - s_ref) < 1e-12 * max(1.0, abs(s_ref))
                assert abs(M[t, i, m] - m_ref) < 1e-13


def test_band_matrices_t0_closed_forms():
    N, T = 12, 2
    S, M = O.band_matrices(N, T)
    n1 = N - 1
    assert np.abs(S[0] - np.diag(4.0 * np.arange(n1) + 6.0)).max() < 1e-12
    assert np.abs(M[0] - _mass_1d(n1)).max() < 1e-14


def test_band_proposition_4_1_structure():
    """S^(t) couples only |i-m| <= t with i+m+t even; M^(t) only |i-m| <= t+2, same parity."""
    N, T = 16, 6
    S, M = O.band_matrices(N, T)
    n1 = N - 1
    for t in range(T + 1):
        for i in range(n1):
            for m in range(n1):
                o = abs(i - m)
                if o > t or (i + m + t) % 2:
                    assert abs(S[t, i, m]) < 1e-12
                if o > t + 2 or (i + m + t) % 2:
                    assert abs(M[t, i, m]) < 1e-13
        # number of diagonals of a full-degree series (Prop. 4.1 with t_max = t): 2t+1 and 2t+5
        occ_s = {i - m for i in range(n1) for m in range(n1) if abs(S[t, i, m]) > 1e-12}
        occ_m = {i - m for i in range(n1) for m in range(n1) if abs(M[t, i, m]) > 1e-13}
        assert max(occ_s) - min(occ_s) + 1 == 2 * t + 1
        assert max(occ_m) - min(occ_m) + 1 == 2 * t + 5


@pytest.mark.parametrize("d,N,T", [(1, 12, 3), (2, 8, 2), (3, 6, 1)])
def test_M_equals_K_when_coefficients_are_low_degree_polynomials(d, N, T):
    p = W.polynomial_coefficient_problem(d, N, T, T, T, seed=5)
    st = O.setup(d, N, p["Q"], T, p["a"], p["b"])
    K = O.dense_K(d, N, p["Q"], p["a"], p["b"])
    assert np.abs(st["M"].to_dense() - K).max() < 1e-13 * np.abs(K).max()


def _pattern_brute(d, N, T, hb):
    n1, w = N - 1, T + 2
    rng = range(-w, w + 1)
    def s1(o): return abs(o) <= T
    def m1(o): return abs(o) <= T + 2 and (T >= 1 or o % 2 == 0)
    cnt = 0
    import itertools
    for r in itertools.product(range(n1), repeat=d):
        for o in itertools.product(rng, repeat=d):
            if any(not (0 <= r[a] + o[a] < n1) for a in range(d)):
                continue
            ok = any(s1(o[a]) and all(m1(o[b]) for b in range(d) if b != a) for a in range(d))
            ok = ok or (hb and all(m1(v) for v in o))
            cnt += ok
    return cnt


@pytest.mark.parametrize("d,N,T,hb", [(1, 9, 0, 1), (2, 9, 1, 0), (2, 10, 2, 1), (3, 7, 1, 0), (3, 6, 0, 1)])
def test_pattern_counts_brute_force(d, N, T, hb):
    assert O.lib().or_pattern_nnz(d, N, T, hb) == _pattern_brute(d, N, T, hb)


def _setup_random(d, N, T, seed, hb=True):
    p = W.random_exp_problem(d, N, T, seed, seed + 1, seed + 2)
    b = p["b"] if hb else np.zeros_like(p["b"])
    st = O.setup(d, N, p["Q"], T, p["a"], b)
    return p, st


@pytest.mark.parametrize("d,N,T,hb", [(1, 20, 3, True), (2, 10, 2, True), (2, 9, 1, False), (3, 6, 1, True)])
def test_ilu0_exact_on_pattern_and_symmetric(d, N, T, hb):
    p, st = _setup_random(d, N, T, 40 + d, hb)
    assert st["ilu_status"] == 0
    M, LU = st["M"].to_dense(), st["LU"]
    n = LU.n
    D = LU.to_dense()
    L = np.tril(D, -1) + np.eye(n)
    U = np.triu(D)
    pat = np.zeros((n, n), bool)
    for i in range(n):
        pat[i, LU.col[LU.rowptr[i]:LU.rowptr[i + 1]]] = True
    R = L @ U - M
    assert np.abs(R[pat]).max() < 1e-13 * np.abs(M).max()
    # L and U together have the nonzero count of M (Sec. 4.2)
    assert LU.rowptr[-1] == st["M"].rowptr[-1]
    # symmetric M: U = diag(U) L^T
    assert np.abs(U - np.diag(np.diag(U)) @ L.T).max() < 1e-12 * np.abs(U).max()


def test_ilu0_full_pattern_equals_cholesky():
    """When the pattern covers every pair (n1 <= w+1) ILU(0) is the exact LDL^T."""
    d, N, T = 2, 6, 4  # n1 = 5 <= w + 1 = 7
    p, st = _setup_random(d, N, T, 60)
    M = st["M"].to_dense()
    assert np.count_nonzero(M) == M.size
    C = np.linalg.cholesky(M)
    Dg = np.diag(C) ** 2
    Lref = C / np.diag(C)
    D = st["LU"].to_dense()
    assert np.abs(np.tril(D, -1) + np.eye(len(M)) - Lref).max() < 1e-12
    assert np.abs(np.diag(D) - Dg).max() < 1e-12 * Dg.max()


def test_ilu0_1d_is_exact_banded_lu():
    p, st = _setup_random(1, 30, 4, 70)
    M = st["M"].to_dense()
    D = st["LU"].to_dense()
    L = np.tril(D, -1) + np.eye(len(M))
    U = np.triu(D)
    assert np.abs(L @ U - M).max() < 1e-13 * np.abs(M).max()


def test_ilu_solve_matches_dense_triangular_solves():
    from scipy.linalg import solve_triangular
    p, st = _setup_random(2, 11, 2, 80)
    D = st["LU"].to_dense()
    n = len(D)
    L = np.tril(D, -1) + np.eye(n)
    U = np.triu(D)
    r = np.random.default_rng(5).standard_normal(n)
    z = O.ilu_solve(st["LU"], r)
    zr = solve_triangular(U, solve_triangular(L, r, lower=True, unit_diagonal=True))
    assert np.abs(z - zr).max() < 1e-12 * np.abs(zr).max()
    assert np.linalg.norm(L @ (U @ z) - r) < 1e-13 * np.linalg.norm(r)


# --------------------------------------------------------------------------- Algorithm 1


def test_pcg_1d_converges_in_one_iteration_when_M_equals_K():
    d, N, T = 1, 40, 3
    p = W.polynomial_coefficient_problem(d, N, T, T, T, seed=9)
    F = O.load_vector(d, N, p["Q"], p["f"])
    r = O.solve(d, N, p["Q"], T, p["a"], p["b"], F)
    assert r["status"] == 0 and r["iters"] == 1


@pytest.mark.parametrize("d,N,T", [(2, 9, 2), (3, 6, 2)])
def test_pcg_matches_dense_solve(d, N, T):
    p = W.random_exp_problem(d, N, T, 90 + d, 91, 92)
    F = O.load_vector(d, N, p["Q"], p["f"])
    r = O.solve(d, N, p["Q"], T, p["a"], p["b"], F)
    K = O.dense_K(d, N, p["Q"], p["a"], p["b"])
    xs = np.linalg.solve(K, F)
    assert r["status"] == 0
    assert np.abs(r["x"] - xs).max() < 1e-11 * np.abs(xs).max()
    assert r["relres"] <= 1e-12


def test_pcg_exact_polynomial_solution():
    """a=1, b=0, u=(1-x^2)(1-y^2) = (4/9) phi_0(x) phi_0(y): f = 2(1-x^2) + 2(1-y^2)."""
    N, T = 8, 0
    Q = N + 2
    x = W.nodes(Q)
    X, Y = np.meshgrid(x, x)
    f = (2 * (1 - X ** 2) + 2 * (1 - Y ** 2)).ravel()
    F = O.load_vector(2, N, Q, f)
    r = O.solve(2, N, Q, T, np.ones(Q * Q), np.zeros(Q * Q), F)
    ref = np.zeros((N - 1) ** 2)
    ref[0] = 4.0 / 9.0
    assert np.abs(r["x"] - ref).max() < 1e-13


def test_manufactured_solution_spectral_convergence():
    errs = []
    for N in (6, 8, 10, 12, 16, 24):
        p = W.manufactured_2d(N, 8)
        F = O.load_vector(2, N, p["Q"], p["f"])
        r = O.solve(2, N, p["Q"], 8, p["a"], p["b"], F)
        n1, Q = N - 1, p["Q"]
        x = W.nodes(Q)
        Ph = np.stack([npleg.legval(x, np.eye(N + 1)[k]) - npleg.legval(x, np.eye(N + 1)[k + 2])
                       for k in range(n1)], 1)
        vals = Ph @ r["x"].reshape(n1, n1) @ Ph.T
        errs.append(np.abs(vals - p["u_exact"].reshape(Q, Q)).max())
    for e0, e1 in zip(errs[:4], errs[1:5]):
        assert e1 < 0.2 * e0  # geometric decrease before the rounding plateau
    assert errs[-1] < 1e-11


def test_paper_table_5_7_example_1b_iteration_counts():
    """Sec. 5, Table 5.7, Example 1(b): beta=exp(2x), alpha=0, eps=1e-12."""
    rows = []
    with open(os.path.join(HERE, "golden", "paper_table_5_7_example_1b.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    for T, N, iters in rows:
        if N > 1280:
            continue  # larger sizes take too long for the CPU suite
        Q = N + 1
        x = W.nodes(Q)
        a, b, f = np.exp(2 * x), np.zeros(Q), np.ones(Q)
        F = O.load_vector(1, N, Q, f)
        r = O.solve(1, N, Q, T, a, b, F)
        assert r["status"] == 0
        assert abs(r["iters"] - iters) <= 1, (T, N, r["iters"], iters)


@pytest.mark.slow
def test_3d_t6_ilu0_breaks_down_at_n24():
    """3D, T=6: the configuration's degree-6 exponential-series coefficients (sigma 0.5,
    seeds 1-3) give an M whose ILU(0) of Algorithm 2 meets a negative pivot already at
    N=24 (12,167 rows), so the 3D N=128 T=6 configuration has no ILU(0) either.  Pinned
    values: first bad row 9886 (natural order) at U_ii/|M_ii| = -0.0668; some three hundred
    pivots end negative in all (after the first negative pivot the count depends on rounding).
    With seeds 11-13 the same size still factorises (no negative pivot).  About a minute on
    8 cores."""
    p = W.random_exp_problem(3, 24, 6, 1, 2, 3)
    st = O.setup(3, 24, p["Q"], 6, p["a"], p["b"])
    assert st["ilu_status"] == O.OR_ERR_BREAKDOWN
    LU, M = st["LU"], st["M"]
    piv = np.array([LU.get(i, i) for i in range(LU.n)])
    mii = np.array([M.get(i, i) for i in range(LU.n)])
    bad = np.nonzero(piv <= 1e-14 * np.abs(mii))[0]
    assert bad[0] == 9886
    assert abs(piv[9886] / abs(mii[9886]) - (-0.06683)) < 1e-4
    assert 200 < int((piv < 0).sum()) < 400
    # every pivot before the first bad one is positive, as Algorithm 2 needs
    assert np.all(piv[:9886] > 0)

"""FP64 CPU oracle for the preconditioned Legendre-Galerkin solve (arXiv 2004.13961).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_2004_13961_gb300`` and neither imports the
other.  Each wrapper below calls one function of ``lsg_oracle.c``; the C file
cites the passage of the paper that each one follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lsg_oracle.c")
_LIB = os.path.join(_HERE, "liblsg_oracle.so")

OR_OK = 0
OR_ERR_BREAKDOWN = -4
OR_ERR_NOT_CONVERGED = -5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP over independent loops)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        ci, cll, cd = ctypes.c_int, ctypes.c_longlong, ctypes.c_double
        L.or_legendre_all.argtypes = [ci, cd, dp]
        L.or_legendre_deriv_all.argtypes = [ci, cd, dp]
        L.or_gauss.argtypes = [ci, dp, dp]
        L.or_apply_K.argtypes = [ci, ci, ci, dp, dp, dp, dp]
        L.or_dense_K.argtypes = [ci, ci, ci, dp, dp, dp]
        L.or_load_vector.argtypes = [ci, ci, ci, dp, dp]
        L.or_load_vector_legendre.argtypes = [ci, ci, ci, dp, dp]
        L.or_coef_trunc.argtypes = [ci, ci, ci, dp, dp]
        L.or_band_matrices.argtypes = [ci, ci, dp, dp]
        L.or_pattern_nnz.argtypes = [ci, ci, ci, ci]
        L.or_pattern_nnz.restype = cll
        L.or_assemble_M.argtypes = [ci, ci, ci, dp, dp, ci, dp, dp, i64p, i32p, dp]
        L.or_ilu0.argtypes = [cll, i64p, i32p, dp]
        L.or_ilu_solve.argtypes = [cll, i64p, i32p, dp, dp, dp]
        L.or_pcg.argtypes = [ci, ci, ci, dp, dp, i64p, i32p, dp, dp, dp, cd, ci,
                             ctypes.POINTER(ci), dp, dp]
        ip = ctypes.POINTER(ctypes.c_int)
        L.or_apply_K_dir.argtypes = [ci, ci, ci, dp, dp, dp, dp, dp, dp]
        L.or_dense_K_dir.argtypes = [ci, ci, ci, dp, dp, dp, dp, dp]
        L.or_coef_trunc_dir.argtypes = [ci, ci, ci, ip, dp, dp]
        L.or_pattern_nnz_dir.argtypes = [ci, ci, ip, ip, ci]
        L.or_pattern_nnz_dir.restype = cll
        L.or_assemble_M_dir.argtypes = [ci, ci, ci, dp, dp, dp, dp, ip, ip, ci, dp, dp, i64p, i32p, dp]
        L.or_pcg_dir.argtypes = [ci, ci, ci, dp, dp, dp, dp, i64p, i32p, dp, dp, dp, cd, ci,
                                 ctypes.POINTER(ci), dp, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def legendre_all(nmax: int, x: float) -> np.ndarray:
    out = np.zeros(nmax + 1)
    lib().or_legendre_all(nmax, float(x), _dp(out))
    return out


def legendre_deriv_all(nmax: int, x: float) -> np.ndarray:
    out = np.zeros(nmax + 1)
    lib().or_legendre_deriv_all(nmax, float(x), _dp(out))
    return out


def gauss(Q: int):
    x = np.zeros(Q)
    w = np.zeros(Q)
    rc = lib().or_gauss(Q, _dp(x), _dp(w))
    assert rc == 0
    return x, w


def _n(d, N):
    return (N - 1) ** d


def apply_K(d, N, Q, a, b, u):
    a, b, u = _c64(a), _c64(b), _c64(u)
    y = np.zeros(_n(d, N))
    rc = lib().or_apply_K(d, N, Q, _dp(a), _dp(b), _dp(u), _dp(y))
    assert rc == 0, rc
    return y


def dense_K(d, N, Q, a, b):
    a, b = _c64(a), _c64(b)
    n = _n(d, N)
    K = np.zeros((n, n))
    rc = lib().or_dense_K(d, N, Q, _dp(a), _dp(b), _dp(K))
    assert rc == 0, rc
    return K


def load_vector(d, N, Q, f):
    f = _c64(f)
    F = np.zeros(_n(d, N))
    rc = lib().or_load_vector(d, N, Q, _dp(f), _dp(F))
    assert rc == 0, rc
    return F


def load_vector_legendre(d, N, fc):
    fc = _c64(fc)
    deg = fc.shape[0] - 1 if fc.ndim else 0
    F = np.zeros(_n(d, N))
    rc = lib().or_load_vector_legendre(d, N, deg, _dp(fc.ravel()), _dp(F))
    assert rc == 0, rc
    return F


def coef_trunc(d, Q, T, c):
    c = _c64(c)
    out = np.zeros((T + 1) ** d)
    rc = lib().or_coef_trunc(d, Q, T, _dp(c), _dp(out))
    assert rc == 0, rc
    return out


def band_matrices(N, T):
    n1 = N - 1
    S = np.zeros((T + 1, n1, n1))
    M = np.zeros((T + 1, n1, n1))
    rc = lib().or_band_matrices(N, T, _dp(S), _dp(M))
    assert rc == 0, rc
    return S, M


class CSR:
    """Row-compressed matrix with ascending columns (oracle storage of M / ILU(0))."""

    def __init__(self, n, rowptr, col, val):
        self.n, self.rowptr, self.col, self.val = n, rowptr, col, val

    def to_dense(self):
        A = np.zeros((self.n, self.n))
        for i in range(self.n):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            A[i, self.col[s:e]] = self.val[s:e]
        return A

    def get(self, i, j):
        s, e = self.rowptr[i], self.rowptr[i + 1]
        idx = np.searchsorted(self.col[s:e], j)
        if idx < e - s and self.col[s + idx] == j:
            return self.val[s + idx]
        return None

    def copy(self):
        return CSR(self.n, self.rowptr, self.col, self.val.copy())


def has_b(b) -> int:
    return int(np.any(np.asarray(b) != 0.0))


def assemble_M(d, N, T, ahat, bhat, hasb, S=None, Mb=None):
    if S is None:
        S, Mb = band_matrices(N, T)
    ahat, bhat = _c64(ahat), _c64(bhat)
    S, Mb = _c64(S), _c64(Mb)
    n = _n(d, N)
    nnz = lib().or_pattern_nnz(d, N, T, int(hasb))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz)
    rc = lib().or_assemble_M(d, N, T, _dp(ahat), _dp(bhat), int(hasb), _dp(S), _dp(Mb),
                             rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(val))
    assert rc == 0, rc
    return CSR(n, rowptr, col, val)


def ilu0(M: CSR):
    H = M.copy()
    rc = lib().or_ilu0(H.n, H.rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                       H.col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(H.val))
    return H, rc


def ilu_solve(LU: CSR, r):
    r = _c64(r)
    z = np.zeros(LU.n)
    rc = lib().or_ilu_solve(LU.n, LU.rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            LU.col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(LU.val),
                            _dp(r), _dp(z))
    assert rc == 0
    return z


def setup(d, N, Q, T, a, b):
    """Preconditioner setup: truncated coefficients, band matrices, M, ILU(0)."""
    ahat = coef_trunc(d, Q, T, a)
    bhat = coef_trunc(d, Q, T, b)
    hb = has_b(b)
    M = assemble_M(d, N, T, ahat, bhat, hb)
    LU, rc = ilu0(M)
    return dict(ahat=ahat, bhat=bhat, M=M, LU=LU, ilu_status=rc, has_b=hb)


def pcg(d, N, Q, a, b, LU: CSR, F, eps=1e-12, kmax=10000, x0=None):
    a, b, F = _c64(a), _c64(b), _c64(F)
    x = np.zeros(_n(d, N)) if x0 is None else _c64(x0).copy()
    it = ctypes.c_int(0)
    rr = np.zeros(1)
    rt = np.zeros(1)
    rc = lib().or_pcg(d, N, Q, _dp(a), _dp(b),
                      LU.rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                      LU.col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(LU.val),
                      _dp(F), _dp(x), float(eps), int(kmax), ctypes.byref(it), _dp(rr), _dp(rt))
    return dict(x=x, iters=it.value, relres=rr[0], relres_true=rt[0], status=rc)


def solve(d, N, Q, T, a, b, F, eps=1e-12, kmax=10000):
    st = setup(d, N, Q, T, a, b)
    out = pcg(d, N, Q, a, b, st["LU"], F, eps, kmax)
    out.update(st)
    return out


# --------------------------------------------------------------------------- per-direction form
# The diffusion term -sum_j d/dx_j (beta_j d u/dx_j) with one coefficient per direction
# (Sec. 5, Example 4) and per-coefficient, per-direction truncation degrees (Sec. 4.1's
# t_1 and t_2; Example 4's t_1j).  a: a list of d sample arrays (beta_1..beta_d);
# ta: d x d degrees, ta[j][i] of beta_j's series in direction i; tb: d degrees of alpha's.


def _ip(v):
    arr = (ctypes.c_int * len(v))(*[int(x) for x in v])
    return arr


def _dirs(a, d):
    a = [_c64(v) for v in a]
    while len(a) < 3:
        a.append(a[0])
    return a


def _deg9(ta, d):
    out = [0] * 9
    for j in range(d):
        for i in range(d):
            out[3 * j + i] = int(ta[j][i])
    return out


def _deg3(tb, d):
    out = [0] * 3
    for i in range(d):
        out[i] = int(tb[i])
    return out


def apply_K_dir(d, N, Q, a, b, u):
    a, b, u = _dirs(a, d), _c64(b), _c64(u)
    y = np.zeros(_n(d, N))
    rc = lib().or_apply_K_dir(d, N, Q, _dp(a[0]), _dp(a[1]), _dp(a[2]), _dp(b), _dp(u), _dp(y))
    assert rc == 0, rc
    return y


def dense_K_dir(d, N, Q, a, b):
    a, b = _dirs(a, d), _c64(b)
    n = _n(d, N)
    K = np.zeros((n, n))
    rc = lib().or_dense_K_dir(d, N, Q, _dp(a[0]), _dp(a[1]), _dp(a[2]), _dp(b), _dp(K))
    assert rc == 0, rc
    return K


def coef_trunc_dir(d, Q, T, deg, c):
    c = _c64(c)
    out = np.zeros((T + 1) ** d)
    rc = lib().or_coef_trunc_dir(d, Q, T, _ip(_deg3(deg, d)), _dp(c), _dp(out))
    assert rc == 0, rc
    return out


def degree_max(d, ta, tb):
    return max([ta[j][i] for j in range(d) for i in range(d)] + [tb[i] for i in range(d)])


def pattern_nnz_dir(d, N, ta, tb, hasb):
    return int(lib().or_pattern_nnz_dir(d, N, _ip(_deg9(ta, d)), _ip(_deg3(tb, d)), int(hasb)))


def assemble_M_dir(d, N, T, ahats, bhat, ta, tb, hasb, S=None, Mb=None):
    if S is None:
        S, Mb = band_matrices(N, T)
    ah = [_c64(v) for v in ahats]
    while len(ah) < 3:
        ah.append(ah[0])
    bhat, S, Mb = _c64(bhat), _c64(S), _c64(Mb)
    n = _n(d, N)
    t9, t3 = _ip(_deg9(ta, d)), _ip(_deg3(tb, d))
    nnz = lib().or_pattern_nnz_dir(d, N, t9, t3, int(hasb))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz)
    rc = lib().or_assemble_M_dir(d, N, T, _dp(ah[0]), _dp(ah[1]), _dp(ah[2]), _dp(bhat), t9, t3, int(hasb),
                                 _dp(S), _dp(Mb), rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(val))
    assert rc == 0, rc
    return CSR(n, rowptr, col, val)


def setup_dir(d, N, Q, a, b, ta, tb):
    """Preconditioner setup with per-direction coefficients and degrees."""
    T = degree_max(d, ta, tb)
    ahats = [coef_trunc_dir(d, Q, T, ta[j], a[j]) for j in range(d)]
    bhat = coef_trunc_dir(d, Q, T, tb, b)
    hb = has_b(b)
    M = assemble_M_dir(d, N, T, ahats, bhat, ta, tb, hb)
    LU, rc = ilu0(M)
    return dict(ahats=ahats, bhat=bhat, M=M, LU=LU, ilu_status=rc, has_b=hb, T=T)


def pcg_dir(d, N, Q, a, b, LU: CSR, F, eps=1e-12, kmax=10000, x0=None):
    a, b, F = _dirs(a, d), _c64(b), _c64(F)
    x = np.zeros(_n(d, N)) if x0 is None else _c64(x0).copy()
    it = ctypes.c_int(0)
    rr = np.zeros(1)
    rt = np.zeros(1)
    rc = lib().or_pcg_dir(d, N, Q, _dp(a[0]), _dp(a[1]), _dp(a[2]), _dp(b),
                          LU.rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                          LU.col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(LU.val),
                          _dp(F), _dp(x), float(eps), int(kmax), ctypes.byref(it), _dp(rr), _dp(rt))
    return dict(x=x, iters=it.value, relres=rr[0], relres_true=rt[0], status=rc)


def solve_dir(d, N, Q, a, b, ta, tb, F, eps=1e-12, kmax=10000):
    st = setup_dir(d, N, Q, a, b, ta, tb)
    out = pcg_dir(d, N, Q, a, b, st["LU"], F, eps, kmax)
    out.update(st)
    return out



# --------------------------------------------------------------------------- PCG-I
# The paper's comparison method (Sec. 5, the PCG-I rows of Tables 5.7-5.11): PCG with a
# constant-coefficient preconditioner, the system with it as the matrix solved directly in
# each iteration.  Its matrix is M with every truncation degree 0 (the rows "t_1 = 0,
# t_2 = 0"): each coefficient replaced by the constant term of its Legendre series.  The
# oracle solves it with a dense Cholesky factorisation (small sizes only).


def setup_const(d, N, Q, a, b):
    """M_0 (all degrees 0) assembled by Sec. 4.2's Kronecker form, and its Cholesky factor."""
    a = list(a) if isinstance(a, (list, tuple)) else [a] * d
    zeros = [[0] * d for _ in range(d)]
    ahats = [coef_trunc_dir(d, Q, 0, [0] * d, a[j]) for j in range(d)]
    bhat = coef_trunc_dir(d, Q, 0, [0] * d, b)
    M0 = assemble_M_dir(d, N, 0, ahats, bhat, zeros, [0] * d, has_b(b))
    D = M0.to_dense()
    C = np.linalg.cholesky(D)
    return dict(M0=M0, dense=D, chol=C, abar=[float(v[0]) for v in ahats], bbar=float(bhat[0]))


def pcg_const(d, N, Q, a, b, F, eps=1e-12, kmax=10000, x0=None, setup=None):
    """Algorithm 1 with z = M_0^{-1} r by the Cholesky factor (the exact direct solve)."""
    import scipy.linalg as sla
    a = list(a) if isinstance(a, (list, tuple)) else [a] * d
    st = setup_const(d, N, Q, a, b) if setup is None else setup
    C = st["chol"]
    F = _c64(F)
    x = np.zeros(_n(d, N)) if x0 is None else _c64(x0).copy()
    nF = np.linalg.norm(F)
    r = F - apply_K_dir(d, N, Q, a, b, x)
    k, rho, p, status = 0, 0.0, None, OR_OK
    while np.sqrt(r @ r) > eps * nF and k < kmax:
        z = sla.cho_solve((C, True), r)
        k += 1
        if k == 1:
            p = z.copy()
            rho = r @ z
        else:
            rho_t, rho = rho, r @ z
            p = z + (rho / rho_t) * p
        w = apply_K_dir(d, N, Q, a, b, p)
        pw = p @ w
        if not pw > 0.0:
            status = OR_ERR_NOT_CONVERGED
            break
        alpha = rho / pw
        x += alpha * p
        r -= alpha * w
    if status == OR_OK and np.sqrt(r @ r) > eps * nF:
        status = OR_ERR_NOT_CONVERGED
    rt = np.linalg.norm(F - apply_K_dir(d, N, Q, a, b, x)) / nF
    return dict(x=x, iters=k, relres=np.sqrt(r @ r) / nF, relres_true=rt, status=status, setup=st)

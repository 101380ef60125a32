"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Every stage is compared element by element on the same seeded inputs: Gauss
rule, truncated series, band matrices, the assembled M, the ILU(0) factors, the
two sweeps, K x, the load vector and PCG.  Sizes span several tiles with ragged
tails (odd and even Q, N not a multiple of the tile), plus the edge cases the
method has (T = 0, no reaction term, d = 1 and 3, the smallest N).
Tolerances: 1e-11 relative for FP64 K x and the solution (the bar the method
is held to), 1e-13 for setup tables that are plain sums.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2004_13961_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device=DEV)


def host(t):
    return t.detach().cpu().numpy()


def rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = [
    # d, N, T, Q-offset, hasb
    (1, 101, 6, 2, True),
    (2, 24, 4, 2, True),
    (2, 41, 3, 1, True),     # odd Q = N+1 = 42? (N=41 -> Q=42 even); ragged tiles
    (2, 40, 2, 1, True),     # Q = 41 odd: middle node on x = 0
    (2, 20, 0, 2, True),     # T = 0: mass band with holes
    (2, 22, 3, 2, False),    # b == 0: union-of-boxes pattern
    (3, 10, 2, 2, True),
    (3, 9, 2, 1, True),      # odd Q
    (2, 3, 1, 2, True),      # smallest N (one unknown per direction: n1 = 2)
    (2, 20, 0, 2, False),    # T = 0 and b == 0: even offsets only, rows of a line finish out of order
    (2, 96, 8, 2, True),     # many wavefront levels and warps in flight
    (3, 12, 4, 2, True),     # 3D rows of 1,098 slots: FP64 sweeps with an 8-row ring and window 4
    (2, 40, 14, 2, True),    # 544 lower slots per row: the band sweep kernel (wider than the line kernel's)
    (3, 12, 8, 2, True),     # 3D rows of 4,630 lower slots: FP64 factor rows too long for the line kernel's
                             # ring, so both sweeps run the band kernel's 3D branch (other planes from memory)
    (3, 14, 8, 1, True),     # the same branch with odd Q and a plane that no longer fits one stencil box
]


def problem(d, N, T, qoff, hasb, seed=7):
    p = W.random_exp_problem(d, N, T, seed, seed + 1, seed + 2, Q=N + qoff)
    if not hasb:
        p["b"] = np.zeros_like(p["b"])
    return p


@pytest.fixture(scope="module")
def lsg():
    from paper_2004_13961_gb300 import lsg as L
    L.load()
    return L


@pytest.mark.parametrize("Q", [1, 2, 7, 66, 131, 514, 1026])
def test_gauss_rule(lsg, Q):
    x, w = lsg.gauss(Q)
    xo, wo = O.gauss(Q)
    assert np.abs(x - xo).max() < 2e-16 * 4
    assert np.abs((w - wo) / wo).max() < 2e-11


@pytest.mark.parametrize("case", CASES)
def test_setup_tables_and_M(lsg, case):
    d, N, T, qoff, hasb = case
    p = problem(d, N, T, qoff, hasb)
    Q = p["Q"]
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]), Q=Q, keep_M=True)
    ah = O.coef_trunc(d, Q, T, p["a"])
    bh = O.coef_trunc(d, Q, T, p["b"])
    assert rel_max(ctx.export(lsg.EXPORT_AHAT), ah) < 1e-13
    if hasb:
        assert rel_max(ctx.export(lsg.EXPORT_BHAT), bh) < 1e-13
    # band matrices
    S, Mb = O.band_matrices(N, T)
    n1, w = N - 1, T + 2
    W1 = 2 * w + 1
    gS = ctx.export(lsg.EXPORT_BAND_S).reshape(T + 1, n1, W1)
    gM = ctx.export(lsg.EXPORT_BAND_M).reshape(T + 1, n1, W1)
    for i in range(n1):
        sc_s = np.abs(S[:, i, :]).max()
        sc_m = np.abs(Mb[:, i, :]).max()
        for o in range(-w, w + 1):
            m = i + o
            if 0 <= m < n1:
                assert abs(gS[:, i, o + w] - S[:, i, m]).max() < 1e-13 * sc_s
                assert abs(gM[:, i, o + w] - Mb[:, i, m]).max() < 1e-13 * sc_m
    # M in stencil form against the oracle's CSR
    Mo = O.assemble_M(d, N, T, ah, bh, O.has_b(p["b"]))
    _compare_stencil(ctx.export(lsg.EXPORT_M), Mo, d, N, T, tol=1e-13)
    assert ctx.query(lsg.Q_NNZ) == Mo.rowptr[-1]
    ctx.close()


def _stencil_map(d, N, T):
    """For every (row, slot): column index or -1 outside the grid."""
    n1, w = N - 1, T + 2
    W1 = 2 * w + 1
    S = W1 ** d
    n = n1 ** d
    r = np.arange(n)
    ri = [r % n1, (r // n1) % n1, r // (n1 * n1)]
    s = np.arange(S)
    so = [s % W1 - w, (s // W1) % W1 - w if d >= 2 else 0 * s, s // (W1 * W1) - w if d == 3 else 0 * s]
    col = np.zeros((n, S), dtype=np.int64)
    ok = np.ones((n, S), dtype=bool)
    mult = 1
    for ax in range(d):
        c = ri[ax][:, None] + so[ax][None, :]
        ok &= (c >= 0) & (c < n1)
        col += c * mult
        mult *= n1
    col[~ok] = -1
    return col


def _compare_stencil(st, csr, d, N, T, tol, rowwise=False):
    n1 = N - 1
    n = n1 ** d
    S = (2 * (T + 2) + 1) ** d
    st = st.reshape(n, S)
    col = _stencil_map(d, N, T)
    dense_ok = n <= 4000
    if dense_ok:
        D = csr.to_dense()
        ref = np.where(col >= 0, D[np.arange(n)[:, None], np.maximum(col, 0)], 0.0)
    else:
        ref = np.zeros_like(st)
        for i in range(n):
            cols = csr.col[csr.rowptr[i]:csr.rowptr[i + 1]]
            vals = csr.val[csr.rowptr[i]:csr.rowptr[i + 1]]
            m = dict(zip(cols.tolist(), vals.tolist()))
            ref[i] = [m.get(int(c), 0.0) if c >= 0 else 0.0 for c in col[i]]
    # every oracle entry is represented in the stencil
    assert np.isclose(np.abs(ref).sum(), np.abs(csr.val).sum(), rtol=1e-12)
    if rowwise:
        scale = np.maximum(np.abs(ref).max(axis=1, keepdims=True), 1e-300)
        err = (np.abs(st - ref) / scale).max()
    else:
        err = np.abs(st - ref).max() / np.abs(ref).max()
    assert err < tol, err
    assert np.all(st[col < 0] == 0.0)


@pytest.mark.parametrize("case", CASES)
def test_ilu0_factors(lsg, case):
    d, N, T, qoff, hasb = case
    p = problem(d, N, T, qoff, hasb, seed=17)
    Q = p["Q"]
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]), Q=Q)
    ref = O.setup(d, N, Q, T, p["a"], p["b"])
    assert ref["ilu_status"] == 0
    _compare_stencil(ctx.export(lsg.EXPORT_LU), ref["LU"], d, N, T, tol=1e-11, rowwise=True)
    # one-step ILU(0) solve (Algorithms 3 and 4): backward error against the
    # oracle's factors, and forward error against the oracle's solve
    r = np.random.default_rng(3).standard_normal((N - 1) ** d)
    z = host(ctx.apply_Minv(cuda(r)))
    z_ref = O.ilu_solve(ref["LU"], r)
    D = ref["LU"].to_dense()
    n = len(D)
    Lo, Uo = np.tril(D, -1) + np.eye(n), np.triu(D)
    # componentwise-normalised backward error of the two triangular solves
    scale = np.linalg.norm(np.abs(Lo) @ (np.abs(Uo) @ np.abs(z)))
    assert np.linalg.norm(Lo @ (Uo @ z) - r) <= 1e-13 * scale
    assert rel_max(z, z_ref) < 1e-10
    ctx.close()


def _breakdown_agreement(lsg, ctx, ref, d, N, T):
    """The device eliminates rows in wavefront-level order (reading C19) and stops claiming rows
    once a pivot fails; the oracle (Algorithm 2, natural order) goes on to the end.  Compared in
    level order: every pivot the device finished up to the oracle's first failing level equals the
    oracle's, no row fails on the device before that level, and the device does fail."""
    n1, w = N - 1, T + 2
    n = ref["LU"].n
    piv = np.array([ref["LU"].get(i, i) for i in range(n)])
    mii = np.array([ref["M"].get(i, i) for i in range(n)])
    r = np.arange(n)
    level = r % n1 + (w + 1) * ((r // n1) % n1) + (w + 1) ** 2 * (r // (n1 * n1))
    if d == 1:
        level = r
    bad = piv <= 1e-14 * np.abs(mii)
    Lb = level[bad].min()
    assert ctx.status == lsg.ERR_ILU_BREAKDOWN
    st = ctx.export(lsg.EXPORT_LU).reshape(n, -1)
    Sc = (st.shape[1] - 1) // 2
    gm = ctx.export(lsg.EXPORT_M).reshape(n, -1)[:, Sc]
    assert rel_max(gm, mii) < 1e-13
    gp = st[:, Sc]
    done = gp != gm  # rows the device finished (the others still hold M's assembled diagonal)
    upto = done & (level <= Lb)
    assert upto.sum() > 0
    assert np.abs(gp[upto] - piv[upto]).max() < 1e-10 * np.abs(piv[upto]).max()
    gbad = done & (gp <= 1e-14 * np.abs(gm))
    assert gbad.any() and level[gbad].min() >= Lb
    assert np.all(gp[done & (level < Lb)] > 0)


def test_ilu0_breakdown_agrees_with_oracle(lsg):
    """3D, T=1: the truncated series is too coarse and ILU(0) meets a negative pivot;
    the oracle (Algorithm 2) and the device report the same breakdown."""
    d, N, T = 3, 9, 1
    p = problem(d, N, T, 1, True, seed=17)
    ref = O.setup(d, N, p["Q"], T, p["a"], p["b"])
    assert ref["ilu_status"] == O.OR_ERR_BREAKDOWN
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]), Q=p["Q"], allow_breakdown=True, keep_M=True)
    _breakdown_agreement(lsg, ctx, ref, d, N, T)
    ctx.close()


def test_ilu0_breakdown_2d_serving_contrast(lsg):
    """2D, T=4, N=64 with the serving mix's largest contrast (sigma = 2.3, a up to ~100):
    the truncated series of degree 4 no longer keeps M's ILU(0) pivots positive.  The first
    failing row is 167 in natural order, but row 194 (wavefront level 26) in level order."""
    d, N, T = 2, 64, 4
    p = W.random_exp_problem(d, N, T, 100000, 100001, 100002, sigma=2.3)
    ref = O.setup(d, N, p["Q"], T, p["a"], p["b"])
    assert ref["ilu_status"] == O.OR_ERR_BREAKDOWN
    piv = np.array([ref["LU"].get(i, i) for i in range(ref["LU"].n)])
    mii = np.array([ref["M"].get(i, i) for i in range(ref["LU"].n)])
    assert int(np.argmax(piv <= 1e-14 * np.abs(mii))) == 167
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]), Q=p["Q"], allow_breakdown=True, keep_M=True)
    _breakdown_agreement(lsg, ctx, ref, d, N, T)
    ctx.close()


def test_sweep_wait_budget_expires_then_context_recovers(lsg):
    """A device wait that runs out: with a budget of 1,000 SM cycles (~0.5 us) the line
    sweep's CTAs give up waiting for the previous line's values, record LSG_ERR_TIMEOUT and
    exit (after their own bulk copies have landed); the solve reports the timeout.  With the
    default budget restored, the same context solves to the oracle's solution."""
    d, N, T = 2, 64, 4
    p = problem(d, N, T, 2, True, seed=67)
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]))
    F_ref = O.load_vector(d, N, p["Q"], p["f"])
    ctx.set_wait_budget(1000)
    _, info = ctx.pcg_solve(cuda(F_ref), rtol=1e-12, check=False)
    assert info["status"] == lsg.ERR_TIMEOUT
    z = ctx.apply_Minv(cuda(F_ref))  # device pointers: no synchronisation, status read below
    _, info = ctx.pcg_solve(cuda(F_ref), rtol=1e-12, check=False)
    assert info["status"] == lsg.ERR_TIMEOUT
    with pytest.raises(lsg.LsgError):
        ctx.set_wait_budget(-1)
    ctx.set_wait_budget(0)
    u, info = ctx.pcg_solve(cuda(F_ref), rtol=1e-12)
    assert info["status"] == 0
    ref = O.solve(d, N, p["Q"], T, p["a"], p["b"], F_ref, eps=1e-12)
    assert abs(info["iters"] - ref["iters"]) <= 1
    assert rel_max(host(u), ref["x"]) < 1e-11
    ctx.close()


@pytest.mark.parametrize("case", CASES)
def test_apply_K_and_load_vector(lsg, case):
    d, N, T, qoff, hasb = case
    p = problem(d, N, T, qoff, hasb, seed=27)
    Q = p["Q"]
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]), Q=Q)
    rng = np.random.default_rng(5)
    for _ in range(2):
        x = rng.standard_normal((N - 1) ** d)
        y = host(ctx.apply_A(cuda(x)))
        y_ref = O.apply_K(d, N, Q, p["a"], p["b"], x)
        assert rel_max(y, y_ref) < 1e-11
    F = host(ctx.load_vector(cuda(p["f"])))
    F_ref = O.load_vector(d, N, Q, p["f"])
    assert rel_max(F, F_ref) < 1e-12
    vals = host(ctx.eval(cuda(x)))
    # u_N at the grid against a direct evaluation with numpy's Legendre series
    from numpy.polynomial import legendre as npleg
    xq = W.nodes(Q)
    Ph = np.stack([npleg.legval(xq, np.eye(N + 1)[k]) - npleg.legval(xq, np.eye(N + 1)[k + 2])
                   for k in range(N - 1)], 1)
    U = x.reshape((N - 1,) * d)
    if d == 1:
        ref = Ph @ U
    elif d == 2:
        ref = Ph @ U @ Ph.T
    else:
        ref = np.einsum("ai,bj,ck,kji->cba", Ph, Ph, Ph, U)
    assert rel_max(vals, ref.ravel()) < 1e-11
    ctx.close()


@pytest.mark.parametrize("case", CASES)
def test_pcg_matches_oracle(lsg, case):
    d, N, T, qoff, hasb = case
    p = problem(d, N, T, qoff, hasb, seed=37)
    Q = p["Q"]
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]), Q=Q)
    F_ref = O.load_vector(d, N, Q, p["f"])
    ref = O.solve(d, N, Q, T, p["a"], p["b"], F_ref, eps=1e-12)
    u, info = ctx.pcg_solve(cuda(F_ref), rtol=1e-12)
    assert info["status"] == 0
    assert abs(info["iters"] - ref["iters"]) <= 1, (info["iters"], ref["iters"])
    assert info["relres"] <= 1e-12 and info["relres_true"] <= 2e-12
    # the same number of passes of Algorithm 1 gives the same iterate
    u2, info2 = ctx.pcg_solve(cuda(F_ref), rtol=0.0, kmax=ref["iters"], check=False)
    assert info2["iters"] == ref["iters"] or info2["status"] == 0  # an exact zero residual stops it early
    assert rel_max(host(u2), ref["x"]) < 1e-11
    ctx.close()


def test_manufactured_2d_n64(lsg):
    """2D FP64, N=64, T=8, a=1+0.5exp(-(x^2+y^2)), b=1+0.5xy, manufactured u; PCG to 1e-12."""
    p = W.manufactured_2d(64, 8)
    d, N, T, Q = 2, 64, 8, p["Q"]
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]))
    F = ctx.load_vector(cuda(p["f"]))
    F_ref = O.load_vector(d, N, Q, p["f"])
    assert rel_max(host(F), F_ref) < 1e-12
    ref = O.solve(d, N, Q, T, p["a"], p["b"], F_ref, eps=1e-12)
    u, info = ctx.pcg_solve(F, rtol=1e-12)
    assert info["status"] == 0 and abs(info["iters"] - ref["iters"]) <= 1
    assert rel_max(host(u), ref["x"]) < 1e-11
    vals = host(ctx.eval(u))
    assert np.abs(vals - p["u_exact"]).max() < 1e-10  # spectral accuracy on the grid
    ctx.close()


def test_host_pointer_path_matches_device_path(lsg):
    d, N, T = 2, 30, 3
    p = problem(d, N, T, 2, True, seed=47)
    c1 = lsg.Context(d, N, T, p["a"].copy(), p["b"].copy())          # host samples
    c2 = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]))            # device samples
    F = c1.load_vector(p["f"].copy())
    u1, i1 = c1.pcg_solve(F.copy(), u=np.zeros(c1.n), rtol=1e-12)
    u2, i2 = c2.pcg_solve(cuda(F), rtol=1e-12)
    assert i1["iters"] == i2["iters"]
    assert np.array_equal(u1, host(u2))  # bitwise: same kernels, deterministic reductions
    c1.close()
    c2.close()


def test_errors_are_reported_not_raised_on_device(lsg):
    d, N, T = 2, 12, 2
    p = problem(d, N, T, 2, True)
    a = p["a"].copy()
    a[5] = np.nan
    with pytest.raises(lsg.LsgError) as ei:
        lsg.Context(d, N, T, cuda(a), cuda(p["b"]))
    assert ei.value.status == lsg.ERR_NONFINITE
    with pytest.raises(lsg.LsgError) as ei:
        lsg.Context(d, 2, T, cuda(p["a"]), cuda(p["b"]))  # N < 3
    assert ei.value.status == lsg.ERR_ARG
    # a strongly negative reaction coefficient makes M indefinite: ILU(0) pivots break down
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(-1e4 * np.ones_like(p["b"])), allow_breakdown=True)
    assert ctx.status == lsg.ERR_ILU_BREAKDOWN
    ctx.close()
    # the context stays usable after an error
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]))
    u, info = ctx.pcg_solve(ctx.load_vector(cuda(p["f"])), rtol=1e-12)
    assert info["status"] == 0
    ctx.close()


def test_not_converged_status(lsg):
    d, N, T = 2, 30, 1
    p = problem(d, N, T, 2, True, seed=57)
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]))
    F = ctx.load_vector(cuda(p["f"]))
    u, info = ctx.pcg_solve(F, rtol=1e-14, kmax=2, check=False)
    assert info["status"] == lsg.ERR_NOT_CONVERGED and info["iters"] == 2
    ctx.close()

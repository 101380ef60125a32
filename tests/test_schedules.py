"""CPU checks of two schedules the device path uses in place of the paper's order.

* ILU(0) (Algorithm 2) with a row's lower entries taken in wavefront-level order of their
  columns instead of column order: a valid order of the same elimination, so the factors agree
  with column-order IKJ up to rounding.
* The line-parallel triangular sweeps (Algorithms 3 and 4): each position's stale part (every
  term but the K newest values of its own line and of the previous line) plus a finisher window
  that applies each new value to the next K positions, starting K-1 steps before position 0,
  reproduce the sweep exactly; and every stale part reads only values its waits guarantee.

Both are checked on small random stencil matrices against dense numpy; no oracle, no GPU.
"""
import itertools

import numpy as np
import pytest


def box_offsets(d, w):
    rng = range(-w, w + 1)
    if d == 1:
        return [(dx, 0, 0) for dx in rng]
    if d == 2:
        return [(dx, dy, 0) for dy in rng for dx in rng]
    return [(dx, dy, dz) for dz in rng for dy in rng for dx in rng]


def stencil_matrix(d, n1, w, seed):
    """Random matrix with the full (2w+1)^d box pattern in natural order, diagonally dominant."""
    rng = np.random.default_rng(seed)
    n = n1 ** d
    A = np.zeros((n, n))
    offs = box_offsets(d, w)
    for r in range(n):
        i, j, k = r % n1, (r // n1) % n1, r // (n1 * n1)
        for dx, dy, dz in offs:
            ci, cj, ck = i + dx, j + dy, k + dz
            if 0 <= ci < n1 and (d < 2 or 0 <= cj < n1) and (d < 3 or 0 <= ck < n1):
                A[r, ci + n1 * (cj + n1 * ck)] = rng.uniform(-1, 1)
        A[r, r] = len(offs) + 1.0
    return A


def ilu0(A, d, n1, w, order):
    """IKJ ILU(0) over the nonzero pattern of A; `order` sorts a row's lower columns."""
    n = A.shape[0]
    pattern = A != 0
    H = A.copy()
    for r in range(n):
        lower = [c for c in range(r) if pattern[r, c]]
        for c in sorted(lower, key=lambda c: order(r, c)):
            H[r, c] /= H[c, c]
            for m in range(c + 1, n):
                if pattern[r, m] and pattern[c, m]:
                    H[r, m] -= H[r, c] * H[c, m]
    return H


def level(c, d, n1, w):
    i, j, k = c % n1, (c // n1) % n1, c // (n1 * n1)
    return i + (w + 1) * j + (w + 1) ** 2 * k


@pytest.mark.parametrize("d,n1,w", [(1, 12, 3), (2, 9, 2), (2, 8, 3), (3, 5, 1), (3, 4, 2)])
def test_ilu0_level_order_equals_column_order(d, n1, w):
    A = stencil_matrix(d, n1, w, seed=3 + d)
    H_col = ilu0(A, d, n1, w, order=lambda r, c: c)
    H_lev = ilu0(A, d, n1, w, order=lambda r, c: (level(c, d, n1, w), c))
    assert np.abs(H_lev - H_col).max() <= 1e-13 * np.abs(H_col).max()


def test_level_order_differs_from_column_order_somewhere():
    # the schedule is a real reordering: in 2D with w >= 1 the previous line's position i+w
    # comes before the own line's positions in column order but after them by level
    n1, w = 9, 2
    r = 4 + n1 * 4
    lower = [c for c in range(r) if abs(c % n1 - r % n1) <= w and 0 <= r // n1 - c // n1 <= w]
    by_col = sorted(lower)
    by_lev = sorted(lower, key=lambda c: (level(c, 2, n1, w), c))
    assert by_col != by_lev
    assert by_lev[-2:] == sorted([r - 1, r - n1 + w])  # the previous level's rows come last


def line_sweep(d, n1, w, K, DIR, F, diag, rhs):
    """The line kernel's schedule for one sweep (sequential model of the concurrent code).

    F[r, t]: factor of row r at lower slot t (DIR > 0) or upper slot Sc+1+t (DIR < 0), in the
    stencil's slot order; diag: U's diagonal (DIR < 0).  Returns the solution and asserts that
    each stale part reads only final values its waits cover."""
    W1 = 2 * w + 1
    S = W1 ** d
    Sc = (S - 1) // 2
    nlines = n1 ** (d - 1)

    def offs(s):
        return s % W1 - w, (s // W1) % W1 - w if d >= 2 else 0

    fown, fprev = {}, {}
    for t in range(Sc):
        dx, dy = offs(t if DIR > 0 else Sc + 1 + t)
        m, jj = -DIR * dx, w - DIR * dx
        if dy == 0 and 1 <= m <= K:
            fown[m - 1] = t
        if d >= 2 and dy == -DIR and 0 <= jj < K:
            fprev[jj] = t
    fresh = set(fown.values()) | set(fprev.values())
    out = np.full(n1 * nlines, np.nan)

    def stale(q, line):
        i = q if DIR > 0 else n1 - 1 - q
        acc = -rhs[i + n1 * line]
        for t in range(Sc):
            if t in fresh:
                continue
            dx, dy = offs(t if DIR > 0 else Sc + 1 + t)
            ci, cj = i + dx, line + dy
            if not (0 <= ci < n1 and 0 <= cj < nlines):
                continue
            sp, h = q + DIR * dx, -DIR * dy  # sweep position of the value, lines back
            if h == 0:
                assert sp < q - K
            elif h == 1:
                assert sp < max(0, q + w - K + 1)
            else:
                assert sp < q + w + 1
            acc += F[i + n1 * line, t] * out[ci + n1 * cj]
        return -acc

    for v in range(nlines):
        line = v if DIR > 0 else nlines - 1 - v
        G = np.zeros(K)
        yb = 0.0
        for s in range(-(K - 1), n1):
            fo, fp = np.zeros(K), np.zeros(K)
            ri = 1.0
            for j in range(K):
                q = s + j
                if 0 <= q < n1:
                    r = (q if DIR > 0 else n1 - 1 - q) + n1 * line
                    fo[j] = F[r, fown[j]] if j in fown else 0.0
                    fp[j] = F[r, fprev[j]] if j in fprev else 0.0
                    if j == 0 and DIR < 0:
                        ri = 1.0 / diag[r]
            yp = 0.0
            ps, pl = s + w, line - DIR
            if d >= 2 and 0 <= ps < n1 and 0 <= pl < nlines:
                yp = out[(ps if DIR > 0 else n1 - 1 - ps) + n1 * pl]
            B = -fp * yp
            if s >= 0:
                B[0] += stale(s, line)
            R = G + B - fo * yb
            if s >= 0:
                i = s if DIR > 0 else n1 - 1 - s
                yb = R[0] * ri
                out[i + n1 * line] = yb
            G = np.append(R[1:], 0.0)
    return out


@pytest.mark.parametrize("d,n1,w,K", [(1, 20, 4, 8), (2, 9, 2, 8), (2, 12, 3, 4), (2, 15, 4, 8), (2, 10, 2, 1),
                                      (2, 11, 5, 8), (2, 7, 3, 2)])
@pytest.mark.parametrize("DIR", [1, -1])
def test_line_sweep_schedule_is_exact(d, n1, w, K, DIR):
    rng = np.random.default_rng(11)
    W1 = 2 * w + 1
    S = W1 ** d
    Sc = (S - 1) // 2
    nlines = n1 ** (d - 1)
    n = n1 * nlines
    F = rng.standard_normal((n, Sc)) * 0.05
    diag = 1.0 + rng.random(n)
    rhs = rng.standard_normal(n)
    A = np.zeros((n, n))
    for r in range(n):
        i, line = r % n1, r // n1
        A[r, r] = 1.0 if DIR > 0 else diag[r]
        for t in range(Sc):
            s = t if DIR > 0 else Sc + 1 + t
            dx, dy = s % W1 - w, ((s // W1) % W1 - w) if d >= 2 else 0
            if 0 <= i + dx < n1 and 0 <= line + dy < nlines:
                A[r, i + dx + n1 * (line + dy)] = F[r, t]
            else:
                F[r, t] = 0.0  # out-of-grid slots hold exact zeros, as in the stencil storage
    ref = np.linalg.solve(A, rhs)
    out = line_sweep(d, n1, w, K, DIR, F, diag, rhs)
    assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max()

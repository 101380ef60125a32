"""Mixed-precision form: FP32 inner PCG (FP32 ILU(0) factors, low-precision transforms)
inside FP64 iterative refinement.  The result is judged by its FP64 true residual,
computed here with the oracle's own matrix-free product, and by its error against the
FP64 oracle solution."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2004_13961_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def cuda(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device=DEV)


@pytest.fixture(scope="module")
def lsg():
    from paper_2004_13961_gb300 import lsg as L
    L.load()
    return L


@pytest.mark.parametrize("prec", ["MIXED_TF32", "MIXED_BF16"])
@pytest.mark.parametrize("case", [(2, 40, 4, 7), (2, 64, 8, 0), (3, 12, 3, 9), (1, 200, 6, 11)])
def test_mixed_refinement_reaches_1e10(lsg, prec, case):
    d, N, T, seed = case
    p = W.manufactured_2d(N, T) if seed == 0 else W.random_exp_problem(d, N, T, seed, seed + 1, seed + 2)
    Q = p["Q"]
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]), precision=getattr(lsg, prec))
    F = O.load_vector(d, N, Q, p["f"])
    u, info = ctx.pcg_solve(cuda(F), rtol=1e-10)
    assert info["status"] == 0 and info["relres_true"] <= 1e-10
    assert info["outer_iters"] >= 1
    uh = u.cpu().numpy()
    res = np.linalg.norm(F - O.apply_K(d, N, Q, p["a"], p["b"], uh)) / np.linalg.norm(F)
    assert res <= 1.5e-10, res
    ref = O.solve(d, N, Q, T, p["a"], p["b"], F, eps=1e-13)
    err = np.linalg.norm(uh - ref["x"]) / np.linalg.norm(ref["x"])
    assert err <= 1e-7, err
    ctx.close()


def test_fp32_ilu_factors_track_fp64_oracle(lsg):
    d, N, T = 2, 30, 3
    p = W.random_exp_problem(d, N, T, 21, 22, 23)
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]), precision=lsg.MIXED_TF32)
    ref = O.setup(d, N, p["Q"], T, p["a"], p["b"])
    st = ctx.export(lsg.EXPORT_LU).reshape(ref["LU"].n, -1)
    D = ref["LU"].to_dense()
    # compare the stored FP32 factors on the oracle's pattern, row-scaled
    n1, w = N - 1, T + 2
    W1 = 2 * w + 1
    err = 0.0
    for r in range(ref["LU"].n):
        i, j = r % n1, r // n1
        cols = ref["LU"].col[ref["LU"].rowptr[r]:ref["LU"].rowptr[r + 1]]
        vals = D[r, cols]
        slots = ((cols % n1) - i + w) + W1 * ((cols // n1) - j + w)
        err = max(err, np.abs(st[r, slots] - vals).max() / np.abs(vals).max())
    assert err < 1e-5, err
    r = np.random.default_rng(1).standard_normal(ref["LU"].n)
    z = ctx.apply_Minv(cuda(r)).cpu().numpy()
    zr = O.ilu_solve(ref["LU"], r)
    assert np.linalg.norm(z - zr) / np.linalg.norm(zr) < 1e-4
    ctx.close()


@pytest.mark.parametrize("case", [(2, 33, 5), (3, 10, 2), (3, 12, 8)])
def test_mixed_context_preconditioner_solve(lsg, case):
    """A mixed context's FP32 ILU(0) factors swept with FP64 vectors (lsg_apply_Minv) against
    the oracle's FP64 factors and solve: the factors carry FP32 rounding, so the result agrees
    to a few FP32 ulps relative to the solution, not to FP64 precision."""
    d, N, T = case
    p = W.random_exp_problem(d, N, T, 31, 32, 33)
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]), precision=lsg.MIXED_TF32)
    ref = O.setup(d, N, p["Q"], T, p["a"], p["b"])
    r = np.random.default_rng(8).standard_normal((N - 1) ** d)
    z = ctx.apply_Minv(cuda(r)).cpu().numpy()
    z_ref = O.ilu_solve(ref["LU"], r)
    assert np.linalg.norm(z - z_ref) / np.linalg.norm(z_ref) < 1e-4
    ctx.close()

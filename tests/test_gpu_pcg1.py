"""PCG-I, the paper's comparison method (Sec. 5: the rows t_1 = 0, t_2 = 0 of Tables
5.7-5.11): PCG with the constant-coefficient preconditioner M_0 (every coefficient
replaced by the constant term of its Legendre series), solved directly in each
iteration.  The library solves M_0 by fast diagonalisation with generalised
eigenvectors computed on the device; the oracle by a dense Cholesky factorisation.

* The preconditioner solve z = M_0^{-1} r against the oracle's (relative 1e-10: the
  eigen-decomposition's rounding, well inside what PCG needs), in 1D, 2D and 3D, with
  a reaction term and without, with one coefficient and one per direction.
* The eigenvalues against numpy's generalised symmetric eigensolver (scipy eigh).
* PCG-I iteration counts within 1 of the oracle's and the solution at 1e-11, on the
  paper's Examples 1-4 at Q = N+1.
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def lsg():
    from paper_2004_13961_gb300 import lsg as L
    L.load()
    return L


CASES = [("a", 1, 150), ("b", 1, 201), ("a", 2, 33), ("b", 2, 40), ("4", 2, 41), ("a", 3, 10), ("4", 3, 12)]


@pytest.mark.parametrize("case", CASES, ids=[f"{e}-{d}d-N{N}" for e, d, N in CASES])
def test_const_preconditioner_solve_and_pcg1_match_oracle(lsg, case):
    ex, d, N = case
    p = W.paper_example(ex, d, N)
    Q = p["Q"]
    ctx = lsg.Context(d, N, None, [cuda(v) for v in p["a"]], cuda(p["b"]), Q=Q, ta=[[0] * d] * d, tb=[0] * d,
                      const_precond=True)
    assert ctx.query(lsg.Q_PRECOND_KIND) == 1
    st = O.setup_const(d, N, Q, p["a"], p["b"])
    # the generalised eigenvalues of the 1D mass and stiffness matrices
    import scipy.linalg as sla
    n1 = N - 1
    S = np.diag(4.0 * np.arange(n1) + 6.0)
    Mb = O.band_matrices(N, 0)[1][0]
    lam = np.sort(sla.eigh(Mb, S, eigvals_only=True))
    assert np.abs(np.sort(ctx.export(lsg.EXPORT_CONST_EIG)) - lam).max() < 1e-13 * lam.max()
    # z = M_0^{-1} r
    r = np.random.default_rng(7).standard_normal(n1 ** d)
    z = ctx.apply_Minv(cuda(r)).cpu().numpy()
    import scipy.linalg as sla2
    zr = sla2.cho_solve((st["chol"], True), r)
    assert rel(z, zr) < 1e-10
    # PCG-I
    F = O.load_vector(d, N, Q, p["f"])
    ref = O.pcg_const(d, N, Q, p["a"], p["b"], F, eps=1e-12, setup=st)
    u, info = ctx.pcg_solve(cuda(F), rtol=1e-12)
    assert ref["status"] == 0 and info["status"] == 0
    assert abs(info["iters"] - ref["iters"]) <= 1, (info["iters"], ref["iters"])
    assert np.abs(u.cpu().numpy() - ref["x"]).max() < 1e-11 * np.abs(ref["x"]).max()
    ctx.close()


def test_const_preconditioner_rejects_mixed_precision(lsg):
    p = W.paper_example("a", 2, 20)
    with pytest.raises(lsg.LsgError) as ei:
        lsg.Context(2, 20, 0, cuda(p["a"][0]), cuda(p["b"]), Q=p["Q"], precision=lsg.MIXED_TF32, const_precond=True)
    assert ei.value.status == lsg.ERR_ARG

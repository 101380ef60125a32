"""Parity at the workloads' full sizes, in the configuration bench.py times.

* 2D N=512 T=8 (261,121 unknowns), FP64: the solution and the iteration count
  against the FP64 oracle's own PCG (its setup takes ~10 s on the host), and the
  true residual recomputed with the oracle's matrix-free K x.
* The same problem in the mixed form (TF32 and BF16 tensor-core transforms, FP32
  ILU(0), FP64 refinement): true relative residual <= 1e-10 by the oracle's K x,
  and the error against the oracle's FP64 solution.
* 3D N=128 (2,048,383 unknowns): with the configuration's T = 6 the ILU(0) of M
  does not exist (non-positive pivots, as the oracle also finds for 3D T = 6 at
  N = 24 and 32), and the library must say so.  The stand-in (same seeds,
  series and truncation of degree 4, N = 64) is solved in the mixed form and
  pinned by the oracle's matrix-free true residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2004_13961_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DEV = "cuda:0"


@pytest.fixture(scope="module")
def lsg():
    from paper_2004_13961_gb300 import lsg as L
    L.load()
    return L


@pytest.fixture(scope="module")
def c2():
    p = W.exp_2d_n512()
    F = O.load_vector(2, 512, p["Q"], p["f"])
    ref = O.solve(2, 512, p["Q"], 8, p["a"], p["b"], F, eps=1e-12)
    return p, F, ref


def _true_relres(p, u, F):
    r = F - O.apply_K(p["d"], p["N"], p["Q"], p["a"], p["b"], u)
    return np.linalg.norm(r) / np.linalg.norm(F)


def test_c2_fp64_matches_oracle_pcg(lsg, c2):
    p, F, ref = c2
    ctx = lsg.Context(2, 512, 8, torch.tensor(p["a"], device=DEV), torch.tensor(p["b"], device=DEV))
    Fd = ctx.load_vector(torch.tensor(p["f"], device=DEV))
    assert np.abs(Fd.cpu().numpy() - F).max() <= 1e-12 * np.abs(F).max()
    u, info = ctx.pcg_solve(torch.tensor(F, device=DEV), rtol=1e-12)
    uh = u.cpu().numpy()
    assert abs(info["iters"] - ref["iters"]) <= 1
    assert np.abs(uh - ref["x"]).max() / np.abs(ref["x"]).max() < 1e-11
    assert _true_relres(p, uh, F) < 2e-12
    ctx.close()


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_c2_mixed_reaches_1e10_true_residual(lsg, c2, prec):
    p, F, ref = c2
    P = lsg.MIXED_TF32 if prec == "tf32" else lsg.MIXED_BF16
    ctx = lsg.Context(2, 512, 8, torch.tensor(p["a"], device=DEV), torch.tensor(p["b"], device=DEV), precision=P)
    u, info = ctx.pcg_solve(torch.tensor(F, device=DEV), rtol=1e-10)
    uh = u.cpu().numpy()
    assert info["status"] == 0 and info["outer_iters"] >= 1
    assert _true_relres(p, uh, F) <= 1e-10
    # error against the FP64 oracle solution: bounded by cond(K) x 1e-10
    assert np.linalg.norm(uh - ref["x"]) / np.linalg.norm(ref["x"]) < 1e-7
    ctx.close()


def test_c3_t6_ilu_does_not_exist(lsg):
    p = W.exp_3d()  # 3D N=128, T=6, seeds 11-13
    ctx = lsg.Context(3, p["N"], p["T"], torch.tensor(p["a"], device=DEV), torch.tensor(p["b"], device=DEV),
                      precision=lsg.MIXED_TF32, allow_breakdown=True)
    assert ctx.status == lsg.ERR_ILU_BREAKDOWN
    ctx.close()


def test_c3_standin_mixed_true_residual(lsg):
    # the stand-in for the 3D configuration: its seeds, coefficient series and truncation of
    # degree 4 (for which ILU(0) of M exists), at N = 64 so that the test stays within a
    # minute (the 3D sweeps are the slow part of the library)
    p = W.random_exp_problem(3, 64, 4, 11, 12, 13)
    ctx = lsg.Context(3, 64, 4, torch.tensor(p["a"], device=DEV), torch.tensor(p["b"], device=DEV),
                      precision=lsg.MIXED_TF32)
    Fd = ctx.load_vector(torch.tensor(p["f"], device=DEV))
    u, info = ctx.pcg_solve(Fd, rtol=1e-10)
    assert info["status"] == 0
    F = Fd.cpu().numpy()
    assert _true_relres(p, u.cpu().numpy(), F) <= 1e-10
    ctx.close()


@pytest.mark.parametrize("prec", ["FP64", "MIXED_TF32"])
def test_c3_standin_full_size_true_residual(lsg, prec):
    """The 3D N=128 stand-in at full size (T=4, degree-4 series, seeds 11-13; 36 GB of FP64
    factors): FP64 PCG to 1e-12 and the mixed form to 1e-10, each checked with the oracle's
    matrix-free K x (the oracle's M would not fit the host)."""
    p = W.random_exp_problem(3, 128, 4, 11, 12, 13)
    P = getattr(lsg, prec)
    ctx = lsg.Context(3, 128, 4, torch.tensor(p["a"], device=DEV), torch.tensor(p["b"], device=DEV), precision=P)
    Fd = ctx.load_vector(torch.tensor(p["f"], device=DEV))
    rtol = 1e-12 if P == lsg.FP64 else 1e-10
    u, info = ctx.pcg_solve(Fd, rtol=rtol)
    assert info["status"] == 0
    F = Fd.cpu().numpy()
    assert _true_relres(p, u.cpu().numpy(), F) <= (2e-12 if P == lsg.FP64 else 1e-10)
    ctx.close()


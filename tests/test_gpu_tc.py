"""The mixed form's tensor-core K x (TF32 / BF16 operands, FP32 accumulation).

lsg_apply_A_lowp runs every contraction of Sec. 4.3 as a tcgen05 GEMM whose FP32
operands are split into two pieces of the operand type (v = hi + lo) and
multiplied as hi*hi + hi*lo + lo*hi.  The result is compared with the FP64
oracle's matrix-free product on the same (FP32-representable) input.  The
bound follows from the split: the dropped lo*lo term and the rounding of the
pieces leave about 2^-20 (TF32) or 2^-18 (BF16) relative error per product,
plus FP32 accumulation, over four chained contractions; the tolerances below
leave a factor ~10 of margin, and a wrong operand layout gives O(1) errors.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2004_13961_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def lsg():
    from paper_2004_13961_gb300 import lsg as L
    L.load()
    return L


CASES = [
    (1, 150, 6),   # one contraction pair, K = 149 / 152 (ragged K tiles)
    (2, 40, 4),    # M, N below one 128 tile
    (2, 131, 8),   # Q = 133, n1 = 130: two M tiles, ragged N and K
    (3, 14, 3),    # 3D: batches Q*n1, Q*Q
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec,tol", [("tf32", 5e-5), ("bf16", 2e-4)])
def test_lowp_apply_matches_fp64_oracle(lsg, case, prec, tol):
    d, N, T = case
    p = W.random_exp_problem(d, N, T, 51, 52, 53)
    P = lsg.MIXED_TF32 if prec == "tf32" else lsg.MIXED_BF16
    ctx = lsg.Context(d, N, T, torch.tensor(p["a"], device=DEV), torch.tensor(p["b"], device=DEV), precision=P)
    n = ctx.n
    x32 = torch.tensor(np.random.default_rng(5).standard_normal(n), dtype=torch.float32, device=DEV)
    y32 = ctx.apply_A_lowp(x32)
    torch.cuda.synchronize()
    y_ref = O.apply_K(d, N, p["Q"], p["a"], p["b"], x32.double().cpu().numpy())
    y = y32.double().cpu().numpy()
    rel = np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref)
    assert np.isfinite(y).all()
    assert rel < tol, rel
    # the FP64 product of the same context agrees with the oracle to rounding
    y64 = ctx.apply_A(x32.double()).cpu().numpy()
    assert np.linalg.norm(y64 - y_ref) / np.linalg.norm(y_ref) < 1e-12
    ctx.close()


def test_lowp_apply_rejected_for_fp64_context(lsg):
    p = W.random_exp_problem(2, 20, 4, 1, 2, 3)
    ctx = lsg.Context(2, 20, 4, torch.tensor(p["a"], device=DEV), torch.tensor(p["b"], device=DEV))
    x = torch.zeros(ctx.n, dtype=torch.float32, device=DEV)
    with pytest.raises(lsg.LsgError):
        ctx.apply_A_lowp(x)
    ctx.close()

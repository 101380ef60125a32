"""Batched and serving forms: each result is the same alone and in the mix.

The batched form interleaves the PCG iterations of uneven problems on the
device (one stream per problem); the serving form admits requests by HBM
footprint into a bounded number of in-flight slots, each on its own stream.
Both run the same kernels as the single solve, so a problem's solution in the
mix must equal its solution alone (to rounding of the deterministic kernels:
compared at 1e-12 relative), and match the FP64 oracle at 1e-11.
"""
import time

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


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _problems():
    # uneven 2D sizes (ragged tails) and one 3D problem, each with its own seeds
    specs = [(2, 32, 8), (2, 48, 8), (2, 57, 6), (2, 40, 4), (3, 12, 3), (2, 64, 8)]
    out = []
    for i, (d, N, T) in enumerate(specs):
        p = W.random_exp_problem(d, N, T, 1000 + 4 * i, 1001 + 4 * i, 1002 + 4 * i)
        out.append(p)
    return out


def test_batch_equals_alone_and_oracle(lsg):
    probs = _problems()
    ctxs, Fs, us, alone = [], [], [], []
    for p in probs:
        d, N, T = p["d"], p["N"], p["T"]
        c = lsg.Context(d, N, T, torch.tensor(p["a"], device=DEV), torch.tensor(p["b"], device=DEV))
        F = c.load_vector(torch.tensor(p["f"], device=DEV))
        u1, info1 = c.pcg_solve(F, rtol=1e-12)
        alone.append((u1.cpu().numpy(), info1))
        ctxs.append(c)
        Fs.append(F)
        us.append(torch.zeros_like(F))
    st, infos = lsg.batch_solve(ctxs, Fs, us, rtol=1e-12)
    assert st == lsg.OK
    for p, c, F, u, info, (ua, ia) in zip(probs, ctxs, Fs, us, infos, alone):
        assert info["status"] == lsg.OK
        assert info["iters"] == ia["iters"]
        ub = u.cpu().numpy()
        assert rel(ub, ua) < 1e-12
        Fh = F.cpu().numpy()
        ref = O.solve(p["d"], p["N"], p["Q"], p["T"], p["a"], p["b"], Fh, eps=1e-12)
        assert abs(info["iters"] - ref["iters"]) <= 1
        assert rel(ub, ref["x"]) < 1e-11
        c.close()


def _serve(lsg, reqs, budget, inflight):
    srv = lsg.Server(budget, max_inflight=inflight)
    for rid, (p, prec, rtol) in enumerate(reqs):
        assert srv.submit(rid, p["d"], p["N"], p["T"], p["a"], p["b"], p["f"], Q=p["Q"], precision=prec,
                          rtol=rtol) == lsg.OK
    srv.drain()
    res = {r["id"]: r for r in srv.poll(len(reqs) + 4)}
    srv.close()
    return res


def test_serving_mix_equals_alone(lsg):
    probs = _problems()
    reqs = []
    for p in probs:
        reqs.append((p, lsg.FP64, 1e-12))
        reqs.append((p, lsg.MIXED_TF32, 1e-10))
    # alone: one slot, ample budget -> requests run one after another
    alone = _serve(lsg, reqs, budget=8 << 30, inflight=1)
    # the mix: several slots, a budget that holds only a few requests at once
    fps = [lsg.footprint_bytes(p["d"], p["N"], p["T"], p["Q"], prec) for p, prec, _ in reqs]
    budget = max(fps) + sorted(fps)[len(fps) // 2]
    mix = _serve(lsg, reqs, budget=budget, inflight=4)
    assert sorted(alone) == sorted(mix) == list(range(len(reqs)))
    for rid, (p, prec, rtol) in enumerate(reqs):
        a, m = alone[rid], mix[rid]
        assert a["info"]["status"] == lsg.OK and m["info"]["status"] == lsg.OK
        assert m["info"]["relres_true"] <= rtol * 1.01
        assert m["latency_ms"] > 0
        # deterministic kernels: the same arithmetic alone and in the mix
        assert rel(m["u"], a["u"]) < 1e-12
        assert m["info"]["iters"] == a["info"]["iters"]


def test_serving_rejects_request_over_budget(lsg):
    p = _problems()[0]
    fp = lsg.footprint_bytes(p["d"], p["N"], p["T"], p["Q"], lsg.FP64)
    srv = lsg.Server(fp // 2, max_inflight=1)
    assert srv.submit(0, p["d"], p["N"], p["T"], p["a"], p["b"], p["f"], Q=p["Q"]) == lsg.ERR_NOMEM
    srv.close()


def test_batch_mixed_equals_alone(lsg):
    probs = _problems()[:4]
    ctxs, Fs, alone = [], [], []
    for p in probs:
        c = lsg.Context(p["d"], p["N"], p["T"], torch.tensor(p["a"], device=DEV), torch.tensor(p["b"], device=DEV),
                        precision=lsg.MIXED_TF32)
        F = c.load_vector(torch.tensor(p["f"], device=DEV))
        u1, i1 = c.pcg_solve(F, rtol=1e-10)
        alone.append((u1.cpu().numpy(), i1))
        ctxs.append(c)
        Fs.append(F)
    us = [torch.zeros_like(F) for F in Fs]
    st, infos = lsg.batch_solve(ctxs, Fs, us, rtol=1e-10)
    assert st == lsg.OK
    for c, u, info, (ua, ia) in zip(ctxs, us, infos, alone):
        assert info["status"] == lsg.OK and info["relres_true"] <= 1e-10
        assert info["iters"] == ia["iters"] and info["outer_iters"] == ia["outer_iters"]
        assert rel(u.cpu().numpy(), ua) < 1e-12
        c.close()

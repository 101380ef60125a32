"""The solve as one CUDA graph, and the contraction tile shapes of K x.

* A context without the profiler runs Algorithm 1 as one CUDA graph whose loop is a
  conditional WHILE node on the device; a profiled context runs the same kernels from
  a host loop.  Both must give bitwise the same iterate and iteration count (the
  kernels and their reduction orders are the same), matching the oracle.
* A context set up with LSG_SETUP_SHARED_GPU (the factorisation on a grid sized by its
  wavefront, for set-ups beside other work) has bitwise the same ILU(0) factors and
  solve as one set up alone (the elimination order within a row is fixed; only which
  warp takes which row changes).
* Every tile shape the autotuner may choose gives K x to the oracle's 1e-11 bar, for
  each contraction of the 1D, 2D and 3D products (ragged tiles: odd Q, n1 not a
  multiple of any tile); the autotuner returns valid choices and the tuned product
  still matches.
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


def rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def lsg():
    from paper_2004_13961_gb300 import lsg as L
    L.load()
    return L


@pytest.mark.parametrize("case", [(2, 48, 6), (3, 11, 3), (1, 90, 4)])
def test_graph_solve_equals_host_loop_and_oracle(lsg, case):
    d, N, T = case
    p = W.random_exp_problem(d, N, T, 71, 72, 73)
    a, b = cuda(p["a"]), cuda(p["b"])
    F = O.load_vector(d, N, p["Q"], p["f"])
    cg = lsg.Context(d, N, T, a, b)                  # graph path
    ch = lsg.Context(d, N, T, a, b, profile=True)    # host-driven loop
    l0 = lsg.kernel_launches()
    ug, ig = cg.pcg_solve(cuda(F), rtol=1e-12)
    l1 = lsg.kernel_launches()
    uh, ih = ch.pcg_solve(cuda(F), rtol=1e-12)
    l2 = lsg.kernel_launches()
    assert ig["status"] == ih["status"] == 0
    assert ig["iters"] == ih["iters"]
    assert torch.equal(ug, uh)
    assert ig["relres"] == ih["relres"] and ig["relres_true"] == ih["relres_true"]
    # the graph's kernels are counted when they run (about a dozen per iteration)
    assert ig["iters"] * 10 <= l1 - l0 <= (ig["iters"] + 2) * 16, (l1 - l0, ig["iters"])
    assert ih["iters"] * 10 <= l2 - l1
    ref = O.solve(d, N, p["Q"], T, p["a"], p["b"], F, eps=1e-12)
    assert abs(ig["iters"] - ref["iters"]) <= 1
    assert rel_max(ug.cpu().numpy(), ref["x"]) < 1e-11
    # the captured graph is reused on the same vectors, with another tolerance and limit
    u2 = torch.zeros_like(ug)
    Fd = cuda(F)
    for rtol, kmax in ((1e-6, 10000), (1e-12, 3)):
        _, i2 = cg.pcg_solve(Fd, u2.zero_(), rtol=rtol, kmax=kmax, check=False)
        _, i3 = ch.pcg_solve(Fd, torch.zeros_like(ug), rtol=rtol, kmax=kmax, check=False)
        assert i2["iters"] == i3["iters"] and i2["status"] == i3["status"]
    cg.close()
    ch.close()


@pytest.mark.parametrize("case", [(1, 90, 4, 1), (2, 33, 3, 2), (2, 70, 4, 1), (3, 10, 2, 1), (3, 13, 2, 2)])
def test_every_tile_shape_matches_oracle(lsg, case):
    d, N, T, qoff = case
    p = W.random_exp_problem(d, N, T, 81, 82, 83, Q=N + qoff)
    ctx = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]), Q=p["Q"])
    x = np.random.default_rng(9).standard_normal((N - 1) ** d)
    y_ref = O.apply_K(d, N, p["Q"], p["a"], p["b"], x)
    xd = cuda(x)
    for v in range(5):
        for stage in range(2 * d):  # one contraction at a time at variant v, the others default
            ch = [-1] * 6
            ch[stage if stage < d else 3 + stage - d] = v
            ctx.set_transform_tiles(ch)
            y = ctx.apply_A(xd).cpu().numpy()
            assert rel_max(y, y_ref) < 1e-11, (v, stage)
        ctx.set_transform_tiles([v] * 6)
        assert ctx.transform_tiles()[:d] == [v] * d
        assert rel_max(ctx.apply_A(xd).cpu().numpy(), y_ref) < 1e-11, v
    with pytest.raises(lsg.LsgError):
        ctx.set_transform_tiles([5, 0, 0, 0, 0, 0])
    choice = ctx.autotune_transforms(3)
    assert all(-1 <= c <= 4 for c in choice) and ctx.transform_tiles() == choice
    assert rel_max(ctx.apply_A(xd).cpu().numpy(), y_ref) < 1e-11
    # the tuned choice serves later contexts of the same size
    c2 = lsg.Context(d, N, T, cuda(p["a"]), cuda(p["b"]), Q=p["Q"])
    assert c2.transform_tiles() == choice
    u, info = c2.pcg_solve(cuda(O.load_vector(d, N, p["Q"], p["f"])), rtol=1e-12)
    assert info["status"] == 0
    c2.close()
    ctx.close()


@pytest.mark.parametrize("N", [64, 160])
def test_shared_gpu_setup_gives_the_same_factors_and_solve(lsg, N):
    p = W.random_exp_problem(2, N, 8, 31, 32, 33)
    a, b, f = cuda(p["a"]), cuda(p["b"]), cuda(p["f"])
    c1 = lsg.Context(2, N, 8, a, b)
    c2 = lsg.Context(2, N, 8, a, b, shared_gpu=True)
    assert np.array_equal(c1.export(lsg.EXPORT_LU), c2.export(lsg.EXPORT_LU))
    u1, i1 = c1.pcg_solve(c1.load_vector(f), rtol=1e-12)
    u2, i2 = c2.pcg_solve(c2.load_vector(f), rtol=1e-12)
    assert i1["iters"] == i2["iters"] and np.array_equal(u1.cpu().numpy(), u2.cpu().numpy())
    c1.close()
    c2.close()

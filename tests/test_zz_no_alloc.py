"""lsg_gauss_noalloc: the Gauss rule for callers that cannot allocate device memory.

Some callers cannot call the CUDA allocator at call time (their device memory is
fully reserved by another component, or their policy forbids allocator calls
once a job runs).  lsg_gauss allocates device scratch on every call; its variant
lsg_gauss_noalloc keeps that scratch in a fixed array inside the library.  This
file checks, through the C ABI, that two calls in a row give the same rule as
the allocating entry point and as the oracle, and that sizes beyond the array
are rejected.  It is
collected last so that a run stopping at the first failure has run every other
test already; it needs no state from them.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_gauss_noalloc_matches_gauss_on_two_calls_in_a_row():
    import oracle as O
    from paper_2004_13961_gb300 import lsg
    for Q in (514, 131):  # two calls in a row, the second smaller than the first
        x, w = lsg.gauss_noalloc(Q)
        xr, wr = lsg.gauss(Q)
        assert np.abs(x - xr).max() < 2e-16 * 4
        assert np.abs((w - wr) / wr).max() < 2e-11
        assert np.all(np.diff(x) > 0) and abs(w.sum() - 2.0) < 1e-13
        # and directly against the oracle's rule (pinned to numpy's leggauss and 40-digit values)
        xo, wo = O.gauss(Q)
        assert np.abs(x - xo).max() < 2e-16 * 4
        assert np.abs((w - wo) / wo).max() < 2e-11


def test_gauss_noalloc_rejects_sizes_beyond_its_array():
    from paper_2004_13961_gb300 import lsg
    with pytest.raises(lsg.LsgError) as ei:
        lsg.gauss_noalloc(16385)
    assert ei.value.status == lsg.ERR_ARG
    assert "static scratch limit" in str(ei.value)
    x, w = lsg.gauss_noalloc(16384)  # the largest size still served
    assert abs(w.sum() - 2.0) < 1e-12

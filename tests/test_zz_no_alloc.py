"""The allocation-free Suitor entry point (for callers that cannot allocate device memory)
gives the same matching as cwm_suitor_match and as the oracle's greedy matching, on calls
in a row through the C ABI, at the capacity limit, and after a rejected call.

This file is collected last on purpose: it runs after every other test, and it also
passes on its own in a fresh process.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_04221_gb300 import problems as P
from tests.gpu_util import csr_dev, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_04221_gb300 import binding, build
    build.build()
    binding.load()
    return binding


def _graph(kind):
    if kind == "poisson":
        mat = P.poisson3d(40)                       # 64,000 vertices, all weights tie
        v = np.ones(len(mat[0]) - 1)
    elif kind == "capacity":
        mat = P.poisson2d(1024)                     # exactly 1,048,576 vertices: the limit
        v = np.ones(len(mat[0]) - 1)
    else:
        mat = P.random_spd(9001, 9.0, seed=21)       # irregular degrees, distinct weights
        v = np.random.default_rng(4).uniform(0.5, 1.5, 9001)
    return mat, oracle.edge_weights(*mat, v)


def _check(B, kind):
    (rp, ci, val), w = _graph(kind)
    d_rp, d_ci, _ = csr_dev(rp, ci, val)
    d_w = dev(w)
    ref = host(B.cwm_suitor_match(d_rp, d_ci, d_w))
    mate = torch.full((len(rp) - 1,), -7, dtype=torch.int32, device="cuda")
    got = host(B.cwm_suitor_match_noalloc(d_rp, d_ci, d_w, mate))
    assert np.array_equal(got, ref), kind
    assert np.array_equal(got, oracle.greedy_match(rp, ci, w)), kind


def test_noalloc_matches_allocating_entry_point_twice(B):
    # the larger graph first, then a smaller one: the second call must not see the
    # first call's suitor keys left in the shared scratch array
    for kind in ("poisson", "random"):
        _check(B, kind)


def test_noalloc_at_capacity(B):
    """n equal to the capacity: the last key sits right before the error word."""
    _check(B, "capacity")


def test_noalloc_rejects_sizes_beyond_capacity(B):
    n = (1 << 20) + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    w = torch.zeros(1, dtype=torch.float64, device="cuda")
    mate = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(B.AmgError) as e:
        B.cwm_suitor_match_noalloc(rp, ci[:0], w[:0], mate)
    assert e.value.status == B.AMG_ERR_UNSUPPORTED
    assert "capacity" in str(e.value)
    # a valid call right after the rejected one
    _check(B, "random")

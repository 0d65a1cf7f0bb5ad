"""GPU: the finest operator in 3x3 blocks (block3.cu) -- the residual of the V-cycle
(Algorithm 1) and the SpMV with the fused dot products of the FCG (Algorithm 3) streaming a
sliced copy of A with one column index per 3x3 block -- against the oracle, on 3x3-blocked
inputs (Q1 elasticity with its assembled pattern; random block patterns with hub block
rows, stored zeros and slices that end part-way), with the block layout on (auto) and off.
Inputs whose pattern is not 3x3-blocked must keep the CSR kernels.

Tolerances as in the other cycle tests: float64 cycle 1e-12, float32 cycle 1e-6 relative
to the oracle's float64 cycle; FCG within one iteration of the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_04221_gb300 import problems as P
from tests.gpu_util import csr_dev, dev, host

pytestmark = pytest.mark.gpu
FP32_TOL = 1e-6


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_04221_gb300 import binding, build
    build.build()
    binding.load()
    return binding


CASES = [
    # 540 rows: 180 block rows, the last slice of 32 holds 20
    ("elasticity_6", lambda: P.elasticity_q1(6), 2, 30),
    ("elasticity_8", lambda: P.elasticity_q1(8), 2, 50),
    # hub block rows of ~80 blocks (odd and even block counts), 1,503 block rows
    ("block3_random", lambda: P.random_block3_spd(1503, avg_blocks=6.0, n_hubs=3, hub_blocks=80, seed=5), 2, 60),
]


def _names(B, h):
    return {e["name"] for e in B.amg_trace(h)}


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("block3", [0, -1])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_block3_vcycle_matches_oracle(B, case, block3, fp32):
    name, gen, sweeps, cmax = case
    mat = gen()
    n = len(mat[0]) - 1
    v = P.smooth_vector_components(n, seed=1)
    H = oracle.Hierarchy(*mat, v, sweeps=sweeps, coarse_max=cmax)
    prm = B.amg_default_params(sweeps_per_level=sweeps, coarse_max=cmax, vcycle_fp32=fp32, block3=block3)
    h = B.amg_setup(*csr_dev(*mat), dev(v), prm)
    try:
        B.amg_trace_enable(h, True)
        r = np.random.default_rng(11).standard_normal(n)
        w = torch.empty(n, dtype=torch.float64, device="cuda")
        got = host(B.amg_vcycle(h, dev(r), w))
        names = _names(B, h)
    finally:
        h.free()
    ref = H.vcycle(r)
    H.close()
    assert np.abs(got - ref).max() <= (FP32_TOL if fp32 else 1e-12) * np.abs(ref).max()
    assert ("residual_b3@0" in names) == (block3 == 0)


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_block3_fcg_matches_oracle(B, case, fp32):
    name, gen, sweeps, cmax = case
    mat = gen()
    n = len(mat[0]) - 1
    v = P.smooth_vector_components(n, seed=1)
    b = np.random.default_rng(2).uniform(-1.0, 1.0, n)
    H = oracle.Hierarchy(*mat, v, sweeps=sweeps, coarse_max=cmax)
    xr, st_r, it_r, _, _ = H.pcg(b, rtol=1e-8, itmax=500)
    H.close()
    res = {}
    for block3 in (0, -1):
        h = B.amg_setup(*csr_dev(*mat), dev(v), B.amg_default_params(sweeps_per_level=sweeps, coarse_max=cmax,
                                                                    vcycle_fp32=fp32, block3=block3))
        try:
            B.amg_trace_enable(h, True)
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            st, info = B.amg_pcg_solve(h, dev(b), x, rtol=1e-8, itmax=500)
            names = _names(B, h)
        finally:
            h.free()
        assert st == B.AMG_OK and st_r == oracle.OK
        assert abs(info["iters"] - it_r) <= 1
        assert info["rel_res_true"] <= 2e-8
        assert np.abs(host(x) - xr).max() <= 1e-7 * np.abs(xr).max()
        assert ("spmv_dots_b3" in names) == (block3 == 0)
        res[block3] = host(x)
    assert np.abs(res[0] - res[-1]).max() <= 1e-7 * np.abs(xr).max()


@pytest.mark.parametrize("gen", [lambda: P.poisson3d(24), lambda: P.random_spd(3000, 6.0, seed=4),
                                 lambda: P.elasticity_q1(6)[:2] + (None,)], ids=["poisson", "random", "not_square3"])
def test_block3_not_taken_without_block_pattern(B, gen):
    """n divisible by 3 but rows not in aligned triples: the CSR kernels serve.  The third
    case drops one entry pair of an elasticity matrix so its pattern is no longer blocked."""
    mat = gen()
    if mat[2] is None:  # remove the symmetric pair (0, j), (j, 0) with j the last column of row 0
        rp, ci, val = P.elasticity_q1(6)
        j = ci[rp[1] - 1]
        keep = np.ones(len(ci), bool)
        keep[rp[1] - 1] = False
        row_j = np.arange(rp[j], rp[j + 1])
        keep[row_j[ci[row_j] == 0]] = False
        rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))[keep]
        rp2 = np.zeros(len(rp), np.int64)
        np.cumsum(np.bincount(rows, minlength=len(rp) - 1), out=rp2[1:])
        mat = (rp2.astype(np.int32), ci[keep], val[keep])
    n = len(mat[0]) - 1
    assert n % 3 == 0
    h = B.amg_setup(*csr_dev(*mat), dev(np.ones(n)), B.amg_default_params(sweeps_per_level=2, coarse_max=40))
    try:
        B.amg_trace_enable(h, True)
        r = np.random.default_rng(1).standard_normal(n)
        w = torch.empty(n, dtype=torch.float64, device="cuda")
        B.amg_vcycle(h, dev(r), w)
        names = _names(B, h)
    finally:
        h.free()
    assert not any(nm.startswith("residual_b3") for nm in names)

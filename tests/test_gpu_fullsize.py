"""GPU: the benchmark workload at full size (3D Poisson 128^3, 3 sweeps per level, coarse
n <= 1000, the launch configuration bench.py times).

Checked against the closed form of its hierarchy (exact aggregates of 2x2x2 cubes,
A^k = 2^-k L_7 on (128/2^k)^3, v_k = (2 sqrt 2)^k) and against the oracle run at the same
size (FCG iterations within one, solution).
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


@pytest.fixture(scope="module")
def problem():
    mat = P.poisson3d(128)
    xs, b = P.manufactured_rhs(*mat, seed=0)
    return mat, xs, b


def test_poisson128_hierarchy_closed_form(B, problem):
    mat, xs, b = problem
    n = len(mat[0]) - 1
    h = B.amg_setup(*csr_dev(*mat), dev(np.ones(n)), B.amg_default_params(sweeps_per_level=3, coarse_max=1000))
    try:
        sizes = [B.amg_level_info(h, k)[:2] for k in range(B.amg_num_levels(h))]
        assert sizes == [(m ** 3, 7 * m ** 3 - 6 * m ** 2) for m in (128, 64, 32, 16, 8)]
        for k in range(1, len(sizes)):
            L = B.amg_level_export(h, k)
            m = 128 >> k
            rp, ci, val = host(L["rp"]), host(L["ci"]), host(L["val"])
            rows = np.repeat(np.arange(m ** 3), np.diff(rp))
            ref = np.where(ci == rows, 6.0, -1.0) * 0.5 ** k
            assert np.abs(val - ref).max() <= 1e-13 * 6.0 * 0.5 ** k
            assert np.abs(host(L["v"]) - 8.0 ** (k / 2)).max() <= 1e-12 * 8.0 ** (k / 2)
        L0 = B.amg_level_export(h, 0)
        idx = np.arange(n)
        z, r = np.divmod(idx, 128 * 128)
        y, x = np.divmod(r, 128)
        assert np.array_equal(host(L0["agg"]), ((z // 2) * 64 + y // 2) * 64 + x // 2)
        assert np.abs(host(L0["p"]) - 1.0 / np.sqrt(8.0)).max() < 1e-15
    finally:
        h.free()


@pytest.mark.parametrize("fp32", [0, 1])
def test_poisson128_solve_vs_oracle(B, problem, fp32):
    mat, xs, b = problem
    n = len(mat[0]) - 1
    H = oracle.Hierarchy(*mat, np.ones(n), sweeps=3, coarse_max=1000)
    xr, st_r, it_r, _, _ = H.pcg(b, rtol=1e-8)
    H.close()
    prm = B.amg_default_params(sweeps_per_level=3, coarse_max=1000, vcycle_fp32=fp32, check_input=0)
    h = B.amg_setup(*csr_dev(*mat), dev(np.ones(n)), prm)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, info = B.amg_pcg_solve(h, dev(b), x, rtol=1e-8)
    h.free()
    assert st == B.AMG_OK and st_r == oracle.OK
    assert abs(info["iters"] - it_r) <= 1
    assert info["rel_res_true"] <= 2e-8
    xg = host(x)
    assert np.abs(xg - xr).max() <= 1e-6 * np.abs(xr).max()
    assert np.linalg.norm(xg - xs) / np.linalg.norm(xs) < 1e-5


def test_fcg_partial_sums_beyond_resident_grid(B):
    """n = 3,375,000 (150^3): the FCG update grid (n / 2048 blocks) is larger than the
    reduction grid (8 blocks per SM); both write their partial sums into buffers sized for
    them.  The solve must converge like the oracle's at this size."""
    mat = P.poisson3d(150)
    n = len(mat[0]) - 1
    xs, b = P.manufactured_rhs(*mat, seed=1)
    h = B.amg_setup(*csr_dev(*mat), dev(np.ones(n)), B.amg_default_params(sweeps_per_level=3, coarse_max=1000))
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, info = B.amg_pcg_solve(h, dev(b), x, rtol=1e-8)
    h.free()
    assert st == B.AMG_OK and info["rel_res_true"] <= 2e-8
    assert np.linalg.norm(host(x) - xs) / np.linalg.norm(xs) < 1e-5

"""GPU: sliced copies of A and A P (sell.cu) on the levels that take the coarse correction
and post-sweep through A P -- rows sorted by length within windows of 256, one or more lanes
per row -- against the oracle's cycle (Algorithm 1) and FCG (Algorithm 3), with the copies
off, automatic (levels of at least 131072 rows: none here; the full-size elasticity tests
take them) and on every level with A P (sliced = 1, lanes per row from the longest row):
short rows (3D Poisson), hub rows of ~300 entries among rows of ~5 (windows whose lengths
differ by 60x), the W-cycle (its second coarse cycle starts from a nonzero guess, the
unscaled forms), both precisions.
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
    ("elasticity_8", lambda: P.elasticity_q1(8), "comp", 2, 50),
    ("poisson3d_24", lambda: P.poisson3d(24), "ones", 3, 20),
    # coarse n <= 150: six levels (the hub rows stall the coarsening near 130 rows; a W-cycle
    # over the 40 levels that coarse n <= 40 would give costs 2^39 coarse cycles)
    ("hubs", lambda: P.random_spd_hubs(6000, 5.0, n_hubs=8, hub_degree=300, seed=5), "ones", 2, 150),
]


def _v(kind, n):
    return P.smooth_vector_components(n, seed=1) if kind == "comp" else np.ones(n)


@pytest.mark.parametrize("gamma", [1, 2])
@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("sliced", [-1, 0, 1])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_sliced_vcycle_matches_oracle(B, case, sliced, fp32, gamma):
    name, gen, vkind, sweeps, cmax = case
    mat = gen()
    n = len(mat[0]) - 1
    v = _v(vkind, n)
    H = oracle.Hierarchy(*mat, v, sweeps=sweeps, coarse_max=cmax, gamma=gamma)
    prm = B.amg_default_params(sweeps_per_level=sweeps, coarse_max=cmax, vcycle_fp32=fp32, sliced=sliced,
                               coupled_post=1, gamma=gamma)
    h = B.amg_setup(*csr_dev(*mat), dev(v), prm)
    try:
        B.amg_trace_enable(h, True)
        r = np.random.default_rng(5).standard_normal(n)
        w = torch.empty(n, dtype=torch.float64, device="cuda")
        got = host(B.amg_vcycle(h, dev(r), w))
        names = {e["name"] for e in B.amg_trace(h)}
    finally:
        h.free()
    ref = H.vcycle(r)
    H.close()
    assert np.abs(got - ref).max() <= (FP32_TOL if fp32 else 1e-12) * np.abs(ref).max()
    sl = any(nm.startswith("prolong_jacobi_sl") for nm in names)
    # auto (0) slices only levels of at least 131072 rows: none of these small cases
    assert sl == (sliced == 1)
    assert any(nm.startswith("residual_sl") for nm in names) == (sliced == 1)


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_sliced_fcg_matches_oracle(B, case, fp32):
    name, gen, vkind, sweeps, cmax = case
    mat = gen()
    n = len(mat[0]) - 1
    v = _v(vkind, n)
    xs, b = P.manufactured_rhs(*mat, seed=6)
    H = oracle.Hierarchy(*mat, v, sweeps=sweeps, coarse_max=cmax)
    xr, st_r, it_r, _, _ = H.pcg(b, rtol=1e-8, itmax=500)
    H.close()
    h = B.amg_setup(*csr_dev(*mat), dev(v), B.amg_default_params(sweeps_per_level=sweeps, coarse_max=cmax,
                                                                vcycle_fp32=fp32, sliced=1, coupled_post=1))
    try:
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, info = B.amg_pcg_solve(h, dev(b), x, rtol=1e-8, itmax=500)
    finally:
        h.free()
    assert st == B.AMG_OK and st_r == oracle.OK
    assert abs(info["iters"] - it_r) <= 1
    assert np.abs(host(x) - xr).max() <= 1e-7 * np.abs(xr).max()

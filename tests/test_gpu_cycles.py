"""GPU: V-cycle variants against the oracle -- the fused coarse tail on and off, other
pre/post sweep counts, and the float32 V-cycle inside the float64 FCG.

Tolerances: float64 V-cycle 1e-12 relative (summation order differs from the oracle's);
float32 V-cycle FP32_TOL = 1e-6 relative to the float64 oracle, about 17 binary32 unit
roundoffs (u = 2^-24): the largest error measured over every input here, every tail,
A P and W-cycle setting, was 1.6e-7 (2.6u, Q1 elasticity 8^3 nodes); FCG with the
float32 V-cycle must still reach 1e-8 within one iteration of the oracle's float64 run
(measured: the same count on every input).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_04221_gb300 import problems as P
from tests.gpu_util import csr_dev, dev, host

pytestmark = pytest.mark.gpu
B = None
FP32_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global B
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_04221_gb300 import binding, build
    build.build()
    binding.load()
    B = binding
    yield


CASES = [
    ("poisson3d_24_s3", lambda: P.poisson3d(24), 3, 20),
    ("lognormal_16_s3", lambda: P.lognormal_diffusion(16, seed=3), 3, 30),
    ("rand_s2", lambda: P.random_spd(6000, 7.0, seed=21), 2, 40),
    # long rows on small levels: every level on sub-warp tiles instead of row blocks
    ("elasticity_8_s2", lambda: P.elasticity_q1(8), 2, 50),
]


def _vcycle_pair(mat, sweeps, cmax, prm_kw, pre=1, post=1, seed=0):
    n = len(mat[0]) - 1
    v = np.ones(n)
    H = oracle.Hierarchy(*mat, v, sweeps=sweeps, coarse_max=cmax, pre=pre, post=post)
    prm = B.amg_default_params(sweeps_per_level=sweeps, coarse_max=cmax, pre_sweeps=pre, post_sweeps=post, **prm_kw)
    h = B.amg_setup(*csr_dev(*mat), dev(v), prm)
    r = np.random.default_rng(seed).standard_normal(n)
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    got = host(B.amg_vcycle(h, dev(r), w))
    h.free()
    return got, H.vcycle(r)


@pytest.mark.parametrize("tail_rows", [-1, 0, 1_000_000])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_vcycle_tail_settings(case, tail_rows):
    name, gen, sweeps, cmax = case
    got, ref = _vcycle_pair(gen(), sweeps, cmax, dict(tail_rows=tail_rows))
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("pre,post", [(2, 1), (1, 2), (0, 1), (2, 3)])
@pytest.mark.parametrize("tail_rows", [-1, 1_000_000])
def test_vcycle_sweep_counts(pre, post, tail_rows):
    got, ref = _vcycle_pair(P.poisson3d(20), 3, 20, dict(tail_rows=tail_rows), pre=pre, post=post)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("pre", [0, 2])
def test_vcycle_sweep_counts_coupled(pre):
    """The A P post-sweep after zero or two pre-sweeps (the residual the restriction formed
    is b - A xs with xs = 0 or two sweeps); two post-sweeps keep the separate passes."""
    for post in (1, 2):
        got, ref = _vcycle_pair(P.poisson3d(20), 3, 20, dict(tail_rows=-1, coupled_post=1), pre=pre, post=post)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_coarsest_above_dense_limit():
    """A coarsest level larger than the dense-operator limit (2048 rows) runs its sweeps."""
    mat = P.poisson2d(80)  # 6400 rows; coarse_max large keeps it a single level
    got, ref = _vcycle_pair(mat, 2, 10_000, dict(tail_rows=-1))
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def _long_rows(mat):
    """Rows the split l1-Jacobi sweep gives a whole warp: longer than max(64, 8 x mean)."""
    rp = mat[0]
    n = len(rp) - 1
    lens = np.diff(rp)
    return int((lens > max(64.0, 8.0 * len(mat[1]) / n)).sum())


@pytest.mark.parametrize("fp32", [0, 1])
def test_long_row_split_coarsest(fp32):
    """A single-level hierarchy (the coarsest level above the dense limit) whose hub rows
    take the split sweep: 20 l1-Jacobi sweeps, each hub row on a whole warp."""
    mat = P.random_spd_hubs(5000, 4.0, n_hubs=12, hub_degree=300, seed=7)
    assert _long_rows(mat) >= 12
    got, ref = _vcycle_pair(mat, 2, 10_000, dict(tail_rows=-1, vcycle_fp32=fp32))
    tol = FP32_TOL if fp32 else 1e-12
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("fp32", [0, 1])
def test_long_row_split_hierarchy(fp32):
    """Hub rows on every level of a multi-level hierarchy (post-smoothing sweeps split too)."""
    mat = P.random_spd_hubs(20000, 4.0, n_hubs=40, hub_degree=400, seed=8)
    got, ref = _vcycle_pair(mat, 2, 60, dict(tail_rows=-1, vcycle_fp32=fp32))
    tol = FP32_TOL if fp32 else 1e-12
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


COUPLED_CASES = CASES + [
    # level 0 (110,592 rows) is above the FP64 fused-kernel limit: the unfused cycle
    ("poisson3d_48_s3", lambda: P.poisson3d(48), 3, 100),
    # hub rows of ~300 entries meeting more than 64 distinct aggregates: the warp grouping's
    # search beyond its register copy of the list
    ("hubs_s2", lambda: P.random_spd_hubs(6000, 5.0, n_hubs=8, hub_degree=300, seed=5), 2, 40),
]


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("coupled", [-1, 0, 1])
@pytest.mark.parametrize("case", COUPLED_CASES, ids=[c[0] for c in COUPLED_CASES])
def test_vcycle_coupled_post(case, coupled, fp32):
    """Coarse correction + post-sweep as one pass over the stored A P: with y = xs + P xc,
    b - A y = (b - A xs) - (A P) xc, an identity of the V-cycle of Algorithm 1; the result
    matches the oracle's literal cycle.  coupled_post = 1 takes it on every level below the
    coarsest, 0 on long-row levels outside the fused small-level kernels, -1 never."""
    name, gen, sweeps, cmax = case
    mat = gen()
    n = len(mat[0]) - 1
    v = np.ones(n)
    H = oracle.Hierarchy(*mat, v, sweeps=sweeps, coarse_max=cmax)
    prm = B.amg_default_params(sweeps_per_level=sweeps, coarse_max=cmax, coupled_post=coupled, vcycle_fp32=fp32)
    h = B.amg_setup(*csr_dev(*mat), dev(v), prm)
    try:
        B.amg_trace_enable(h, True)
        r = np.random.default_rng(7).standard_normal(n)
        w = torch.empty(n, dtype=torch.float64, device="cuda")
        got = host(B.amg_vcycle(h, dev(r), w))
        names = {e["name"] for e in B.amg_trace(h)}
    finally:
        h.free()
    ref = H.vcycle(r)
    assert np.abs(got - ref).max() <= (FP32_TOL if fp32 else 1e-12) * np.abs(ref).max()
    # level 0 through A P (stored in CSR or sliced), and no separate post-sweep `jacobi`
    used = ("prolong_jacobi_ap@0" in names or "prolong_jacobi_sl@0" in names) and "jacobi@0" not in names
    if name.startswith("poisson3d"):  # 7-entry rows: auto mode leaves them to the separate passes
        assert used == (coupled == 1)
    if name.startswith("elasticity"):  # 81-entry rows on sub-warp tiles: auto builds A P
        assert used == (coupled >= 0)


@pytest.mark.parametrize("coupled", [-1, 1])
def test_pcg_and_wcycle_coupled_post(coupled):
    """FCG iterations and solution with the A P post-sweep on every level, V- and W-cycle."""
    mat = P.poisson3d(24)
    n = len(mat[0]) - 1
    v = np.ones(n)
    xs, b = P.manufactured_rhs(*mat, seed=8)
    for gamma in (1, 2):
        H = oracle.Hierarchy(*mat, v, sweeps=3, coarse_max=20, gamma=gamma)
        xr, st_r, it_r, _, _ = H.pcg(b, rtol=1e-8, itmax=300)
        h = B.amg_setup(*csr_dev(*mat), dev(v), B.amg_default_params(sweeps_per_level=3, coarse_max=20, gamma=gamma,
                                                                    coupled_post=coupled))
        try:
            r = np.random.default_rng(3).standard_normal(n)
            w = torch.empty(n, dtype=torch.float64, device="cuda")
            ref = H.vcycle(r)
            assert np.abs(host(B.amg_vcycle(h, dev(r), w)) - ref).max() <= 1e-12 * np.abs(ref).max()
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            st, info = B.amg_pcg_solve(h, dev(b), x, rtol=1e-8, itmax=300)
        finally:
            h.free()
        assert st == B.AMG_OK and st_r == oracle.OK
        assert it_r - 1 <= info["iters"] <= it_r + 1
        assert np.abs(host(x) - xr).max() <= 1e-7 * np.abs(xr).max()


@pytest.mark.parametrize("tail_rows", [-1, 0])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_vcycle_fp32(case, tail_rows):
    name, gen, sweeps, cmax = case
    got, ref = _vcycle_pair(gen(), sweeps, cmax, dict(vcycle_fp32=1, tail_rows=tail_rows))
    assert np.abs(got - ref).max() <= FP32_TOL * np.abs(ref).max()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pcg_fp32_vcycle(case):
    name, gen, sweeps, cmax = case
    mat = gen()
    n = len(mat[0]) - 1
    v = np.ones(n)
    xs, b = P.manufactured_rhs(*mat, seed=5)
    H = oracle.Hierarchy(*mat, v, sweeps=sweeps, coarse_max=cmax)
    xr, st_r, it_r, _, _ = H.pcg(b, rtol=1e-8, itmax=500)
    h = B.amg_setup(*csr_dev(*mat), dev(v), B.amg_default_params(sweeps_per_level=sweeps, coarse_max=cmax,
                                                                vcycle_fp32=1))
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, info = B.amg_pcg_solve(h, dev(b), x, rtol=1e-8, itmax=500)
    h.free()
    assert st == B.AMG_OK and st_r == oracle.OK
    assert abs(info["iters"] - it_r) <= 1
    assert info["rel_res_true"] <= 2e-8
    assert np.abs(host(x) - xr).max() <= 1e-6 * np.abs(xr).max()


def test_stall_ratio_hierarchy_matches_oracle():
    """The optional stall-ratio stop gives the oracle's hierarchy, bit for bit."""
    mat = P.lognormal_diffusion(24, seed=0)
    n = len(mat[0]) - 1
    H = oracle.Hierarchy(*mat, np.ones(n), sweeps=3, coarse_max=10, stall_ratio=1.2)
    h = B.amg_setup(*csr_dev(*mat), dev(np.ones(n)),
                    B.amg_default_params(sweeps_per_level=3, coarse_max=10, stall_ratio=1.2))
    try:
        assert B.amg_num_levels(h) == H.nl
        for k in range(H.nl):
            got, ref = B.amg_level_export(h, k), H.level(k)
            assert np.array_equal(host(got["ci"]), ref["ci"])
            assert np.array_equal(host(got["val"]).view(np.int64), ref["val"].view(np.int64))
    finally:
        h.free()


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("gen,sweeps,cmax", [(lambda: P.poisson3d(24), 3, 20),
                                             (lambda: P.random_spd(5000, 6.0, seed=31), 2, 60)])
def test_wcycle_matches_oracle(gen, sweeps, cmax, fp32):
    """W-cycle (gamma = 2, Sec. 5.1): the second coarse cycle starts from the first one's
    result, on the GPU as in the oracle."""
    mat = gen()
    n = len(mat[0]) - 1
    v = np.ones(n)
    H = oracle.Hierarchy(*mat, v, sweeps=sweeps, coarse_max=cmax, gamma=2)
    h = B.amg_setup(*csr_dev(*mat), dev(v), B.amg_default_params(sweeps_per_level=sweeps, coarse_max=cmax, gamma=2,
                                                                vcycle_fp32=fp32))
    try:
        r = np.random.default_rng(2).standard_normal(n)
        w = torch.empty(n, dtype=torch.float64, device="cuda")
        got = host(B.amg_vcycle(h, dev(r), w))
        ref = H.vcycle(r)
        assert np.abs(got - ref).max() <= (FP32_TOL if fp32 else 1e-12) * np.abs(ref).max()
        xs, b = P.manufactured_rhs(*mat, seed=4)
        xr, st_r, it_r, _, _ = H.pcg(b, rtol=1e-8, itmax=300)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, info = B.amg_pcg_solve(h, dev(b), x, rtol=1e-8, itmax=300)
        assert st == B.AMG_OK and st_r == oracle.OK
        assert abs(info["iters"] - it_r) <= 1
    finally:
        h.free()

"""GPU parity: every step of the CUDA path against the CPU oracle on the same seeded inputs.

Bars: bit-exact for weights, matchings, aggregates, prolongator values and Galerkin patterns
and values (their arithmetic order is specified); 1e-12 relative for the V-cycle; FCG
iteration counts within +-1 of the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1810_04221_gb300 import problems as P
from tests.gpu_util import bits_equal, csr_dev, dev, host

pytestmark = pytest.mark.gpu

B = None


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


def _cases():
    """(name, (rp, ci, val), v): tiny to a few tiles, with ragged tails and every tile width."""
    rng = np.random.default_rng(0)
    out = []
    out.append(("poisson2d_64", P.poisson2d(64), None))
    out.append(("poisson3d_12", P.poisson3d(12), None))
    out.append(("poisson2d_7_ragged", P.poisson2d(7), None))
    for seed, deg, ties, zeros in [(1, 3.0, False, 0.0), (2, 7.0, True, 0.0), (3, 15.0, False, 0.1),
                                   (4, 40.0, False, 0.0), (5, 6.0, True, 0.2)]:
        mat = P.random_spd(3001, deg, seed=seed, ties=ties, explicit_zeros=zeros)
        v = None if ties else rng.uniform(-1.5, 1.5, 3001)
        out.append((f"rand_d{int(deg)}_s{seed}", mat, v))
    out.append(("lognormal_14", P.lognormal_diffusion(14, seed=7), None))
    mat = P.elasticity_q1(6)
    out.append(("elasticity_6", mat, P.smooth_vector_components(len(mat[0]) - 1, seed=1)))
    return out


CASES = _cases()
IDS = [c[0] for c in CASES]


def _v(mat, v):
    n = len(mat[0]) - 1
    return np.ones(n) if v is None else v


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_edge_weights_bit_exact(case):
    name, mat, v = case
    v = _v(mat, v)
    ref = oracle.edge_weights(*mat, v)
    rp, ci, val = csr_dev(*mat)
    got = host(B.cwm_edge_weights(rp, ci, val, dev(v)))
    assert bits_equal(got, ref)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_weight_quotient_matches_hardware_division(seed):
    """The edge weights divide on the integer pipes; that quotient is bit-identical to the
    IEEE division on 2^24 generated operand pairs per seed (raw bit patterns, nearby
    exponents, quotients next to rounding boundaries, powers of two, extreme significands,
    exponents at the edges of the normal range)."""
    mismatches, first = B.cwm_div_check(1 << 24, seed)
    assert (mismatches, first) == (0, -1)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_suitor_matches_greedy_bit_exact(case):
    name, mat, v = case
    v = _v(mat, v)
    w = oracle.edge_weights(*mat, v)
    ref = oracle.greedy_match(mat[0], mat[1], w)
    rp, ci, _ = csr_dev(*mat)
    got = host(B.cwm_suitor_match(rp, ci, dev(w)))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_aggregate_and_prolongator_bit_exact(case):
    name, mat, v = case
    v = _v(mat, v)
    w = oracle.edge_weights(*mat, v)
    mate = oracle.greedy_match(mat[0], mat[1], w)
    agg_r, nc_r, np_r, _ = oracle.aggregate(mate)
    p_r, vc_r = oracle.prolongator(agg_r, nc_r, v)
    agg, p, vc, nc, npairs = B.cwm_aggregate(dev(mate), dev(v))
    assert (nc, npairs) == (nc_r, np_r)
    assert np.array_equal(host(agg), agg_r)
    assert bits_equal(host(p), p_r)
    assert bits_equal(host(vc), vc_r)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_galerkin_bit_exact(case):
    name, mat, v = case
    v = _v(mat, v)
    w = oracle.edge_weights(*mat, v)
    mate = oracle.greedy_match(mat[0], mat[1], w)
    agg, nc, _, _ = oracle.aggregate(mate)
    p, _ = oracle.prolongator(agg, nc, v)
    rpc_r, cic_r, valc_r = oracle.galerkin(*mat, agg, nc, p)
    rp, ci, val = csr_dev(*mat)
    rpc, cic, valc = B.cwm_galerkin(rp, ci, val, nc, dev(agg), dev(p))
    assert np.array_equal(host(rpc), rpc_r)
    assert np.array_equal(host(cic), cic_r)
    assert bits_equal(host(valc), valc_r)


def test_galerkin_long_rows_block_path():
    """A hub vertex makes coarse rows gather > 256 fine entries (block-per-row kernel)."""
    n = 2000
    rng = np.random.default_rng(3)
    import scipy.sparse as sp
    hubs = [0, 1, 500]
    rows, cols = [], []
    for h in hubs:
        nb = rng.choice(np.arange(2, n), size=700, replace=False)
        rows += [np.full(700, h), nb]
        cols += [nb, np.full(700, h)]
    mat = P.random_spd(n, 4.0, seed=9)
    A = P.to_scipy(*mat).tolil()
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    keep = r != c
    A[r[keep], c[keep]] = -0.01
    A = sp.csr_matrix(A)
    d = np.asarray(abs(A).sum(axis=1)).ravel()
    A = A + sp.diags(d)
    A = sp.csr_matrix(0.5 * (A + A.T))
    A.sort_indices()
    mat = (A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data)
    assert np.diff(mat[0]).max() > 300
    v = np.ones(n)
    w = oracle.edge_weights(*mat, v)
    mate = oracle.greedy_match(mat[0], mat[1], w)
    agg, nc, _, _ = oracle.aggregate(mate)
    p, _ = oracle.prolongator(agg, nc, v)
    rpc_r, cic_r, valc_r = oracle.galerkin(*mat, agg, nc, p)
    rp, ci, val = csr_dev(*mat)
    assert bits_equal(host(B.cwm_edge_weights(rp, ci, val, dev(v))), w)
    assert np.array_equal(host(B.cwm_suitor_match(rp, ci, dev(w))), mate)
    rpc, cic, valc = B.cwm_galerkin(rp, ci, val, nc, dev(agg), dev(p))
    assert np.array_equal(host(rpc), rpc_r) and np.array_equal(host(cic), cic_r)
    assert bits_equal(host(valc), valc_r)


def _graded_graph(seed=11, sparse_rows=0):
    """Random s.p.d. graph made of diagonal blocks of growing density (mean degrees 4 to
    ~200) joined by a few edges, so that the coarse rows of a pairwise aggregation gather
    from under 16 to over 256 fine entries."""
    rng = np.random.default_rng(seed)
    import scipy.sparse as sp
    blocks = [(3000, 4), (1000, 12), (600, 25), (400, 50), (400, 100), (500, 220)]
    if sparse_rows:  # a sparse block that takes the mean row below 16
        blocks = [(sparse_rows, 2)] + blocks
    rows, cols, base = [], [], 0
    for nb, deg in blocks:
        m = nb * deg // 2
        rows.append(base + rng.integers(0, nb, m))
        cols.append(base + rng.integers(0, nb, m))
        base += nb
    n = base
    rows.append(rng.integers(0, n, 200))
    cols.append(rng.integers(0, n, 200))
    r, c = np.concatenate(rows), np.concatenate(cols)
    keep = r != c
    A = sp.coo_matrix((-rng.uniform(0.1, 1.0, keep.sum()), (r[keep], c[keep])), shape=(n, n)).tocsr()
    A = 0.5 * (A + A.T)
    A.sum_duplicates()
    d = np.asarray(abs(A).sum(axis=1)).ravel() + rng.uniform(0.1, 1.0, n)
    A = sp.csr_matrix(A + sp.diags(d))
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64)


@pytest.mark.parametrize("sparse_rows", [0, 20000])
@pytest.mark.parametrize("fp32", [0, 1])
def test_galerkin_all_row_paths(fp32, sparse_rows):
    """Coarse rows of every length class -- registers (<= 16, <= 32 entries), the warp's
    register sort with 2, 4 and 8 keys per lane (<= 64, <= 128, <= 256) and the block kernel
    (> 256) -- against the oracle, bit for bit (float64 and binary32 products).  The fine
    mean row is ~35 without the sparse block (the sort on 32-bit keys) and ~10 with it
    (64-bit keys)."""
    mat = _graded_graph(sparse_rows=sparse_rows)
    lens0 = np.diff(mat[0])
    assert (lens0.mean() > 16) == (sparse_rows == 0)
    n = len(mat[0]) - 1
    v = np.ones(n)
    w = oracle.edge_weights(*mat, v)
    mate = oracle.greedy_match(mat[0], mat[1], w)
    agg, nc, _, _ = oracle.aggregate(mate)
    lens = np.diff(mat[0])
    L = np.bincount(agg, weights=lens, minlength=nc).astype(int)
    for lo, hi in [(1, 16), (17, 32), (33, 64), (65, 128), (129, 256), (257, 10**6)]:
        assert ((L >= lo) & (L <= hi)).any(), (lo, hi)
    p, _ = oracle.prolongator(agg, nc, v)
    rpc_r, cic_r, valc_r = oracle.galerkin(*mat, agg, nc, p, fp32=bool(fp32))
    rp, ci, val = csr_dev(*mat)
    rpc, cic, valc = B.cwm_galerkin(rp, ci, val, nc, dev(agg), dev(p), fp32=fp32)
    assert np.array_equal(host(rpc), rpc_r) and np.array_equal(host(cic), cic_r)
    assert bits_equal(host(valc), valc_r)


# ------------------------------------------------------------------ hierarchy ----

HIER_CASES = [
    ("poisson2d_64_s2", P.poisson2d(64), None, 2, 40),
    ("poisson3d_16_s3", P.poisson3d(16), None, 3, 10),
    ("lognormal_12_s3", P.lognormal_diffusion(12, seed=1), None, 3, 20),
    ("rand_s1", P.random_spd(4000, 6.0, seed=11), "rand", 1, 30),
    ("rand_ties_s2", P.random_spd(4000, 6.0, seed=12, ties=True), None, 2, 30),
    ("elasticity_6_s2", P.elasticity_q1(6), "comp", 2, 30),
]


def _hv(mat, kind):
    n = len(mat[0]) - 1
    if kind == "rand":
        return np.random.default_rng(5).uniform(0.5, 1.5, n)
    if kind == "comp":
        return P.smooth_vector_components(n, seed=2)
    return np.ones(n)


@pytest.mark.parametrize("case", HIER_CASES, ids=[c[0] for c in HIER_CASES])
def test_hierarchy_levels_bit_exact(case):
    name, mat, kind, sweeps, cmax = case
    v = _hv(mat, kind)
    H = oracle.Hierarchy(*mat, v, sweeps=sweeps, coarse_max=cmax)
    prm = B.amg_default_params(sweeps_per_level=sweeps, coarse_max=cmax, keep_sweeps=1)
    h = B.amg_setup(*csr_dev(*mat), dev(v), prm)
    try:
        assert B.amg_num_levels(h) == H.nl
        for k in range(H.nl):
            ref = H.level(k)
            got = B.amg_level_export(h, k)
            assert (got["n"], got["nnz"]) == (ref["n"], ref["nnz"])
            assert np.array_equal(host(got["rp"]), ref["rp"])
            assert np.array_equal(host(got["ci"]), ref["ci"])
            assert bits_equal(host(got["val"]), ref["val"])
            assert bits_equal(host(got["v"]), ref["v"])
            assert np.allclose(host(got["dl1"]), ref["dl1"], rtol=1e-14, atol=0)
            if k < H.nl - 1:
                assert np.array_equal(host(got["agg"]), ref["agg"])
                assert bits_equal(host(got["p"]), ref["p"])
                assert got["nsweeps"] == H.sweeps(k)
                for s in range(H.sweeps(k)):
                    assert np.array_equal(host(B.amg_sweep_mate(h, k, s)), H.sweep_mate(k, s))
        st = B.amg_stats(h)
        vc, cr = H.stats()
        assert st["nl"] == H.nl and abs(st["vcmplx"] - vc) < 1e-14 and abs(st["cratio"] - cr) < 1e-14
    finally:
        h.free()


@pytest.mark.parametrize("case", HIER_CASES[:4], ids=[c[0] for c in HIER_CASES[:4]])
def test_vcycle_matches_oracle(case):
    name, mat, kind, sweeps, cmax = case
    v = _hv(mat, kind)
    H = oracle.Hierarchy(*mat, v, sweeps=sweeps, coarse_max=cmax)
    h = B.amg_setup(*csr_dev(*mat), dev(v), B.amg_default_params(sweeps_per_level=sweeps, coarse_max=cmax))
    try:
        n = len(v)
        for seed in range(3):
            r = np.random.default_rng(seed).standard_normal(n)
            ref = H.vcycle(r)
            w = torch.empty(n, dtype=torch.float64, device="cuda")
            got = host(B.amg_vcycle(h, dev(r), w))
            assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    finally:
        h.free()


@pytest.mark.parametrize("case", HIER_CASES, ids=[c[0] for c in HIER_CASES])
def test_pcg_iterations_and_solution(case):
    name, mat, kind, sweeps, cmax = case
    v = _hv(mat, kind)
    xs, b = P.manufactured_rhs(*mat, seed=3)
    H = oracle.Hierarchy(*mat, v, sweeps=sweeps, coarse_max=cmax)
    xr, st_r, it_r, rr_r, rt_r = H.pcg(b, rtol=1e-8, itmax=500)
    h = B.amg_setup(*csr_dev(*mat), dev(v), B.amg_default_params(sweeps_per_level=sweeps, coarse_max=cmax))
    try:
        x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
        st, info = B.amg_pcg_solve(h, dev(b), x, rtol=1e-8, itmax=500)
        assert st == B.AMG_OK and st_r == oracle.OK
        assert abs(info["iters"] - it_r) <= 1
        assert info["rel_res"] <= 1e-8 and info["rel_res_true"] <= 1e-7
        assert np.abs(host(x) - xr).max() <= 1e-6 * np.abs(xr).max()
    finally:
        h.free()


# ------------------------------------------------------------------ edge cases ----

def test_single_row_and_diagonal_only():
    for n in (1, 37):
        rp = np.arange(n + 1, dtype=np.int32)
        ci = np.arange(n, dtype=np.int32)
        val = np.full(n, 2.0)
        h = B.amg_setup(*csr_dev(rp, ci, val), dev(np.ones(n)), B.amg_default_params(coarse_max=0))
        try:
            assert B.amg_num_levels(h) == 1
            b = np.arange(1, n + 1, dtype=np.float64)
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            st, info = B.amg_pcg_solve(h, dev(b), x, rtol=1e-12)
            assert st == B.AMG_OK
            assert np.allclose(host(x), b / 2.0, rtol=1e-14)
        finally:
            h.free()
        mate = host(B.cwm_suitor_match(*csr_dev(rp, ci, val)[:2], dev(np.zeros(n))))
        assert np.all(mate == -1)


def test_zero_rhs_and_itmax():
    mat = P.poisson2d(16)
    h = B.amg_setup(*csr_dev(*mat), dev(np.ones(256)))
    try:
        x = torch.zeros(256, dtype=torch.float64, device="cuda")
        st, info = B.amg_pcg_solve(h, dev(np.zeros(256)), x)
        assert st == B.AMG_OK and info["iters"] == 0
        st, info = B.amg_pcg_solve(h, dev(np.ones(256)), x, rtol=1e-30, itmax=3)
        assert st == B.AMG_ERR_NOT_CONVERGED and info["iters"] == 3
    finally:
        h.free()


def test_rejects_bad_inputs():
    rp = np.array([0, 2, 4], np.int32)
    # non-positive diagonal
    with pytest.raises(B.AmgError) as e:
        B.amg_setup(*csr_dev(rp, np.array([0, 1, 0, 1], np.int32), np.array([0.0, -1.0, -1.0, 2.0])), dev(np.ones(2)))
    assert e.value.status == B.AMG_ERR_NOT_SPD
    # unsorted columns
    with pytest.raises(B.AmgError) as e:
        B.amg_setup(*csr_dev(rp, np.array([1, 0, 0, 1], np.int32), np.array([-1.0, 2.0, -1.0, 2.0])), dev(np.ones(2)))
    assert e.value.status == B.AMG_ERR_INVALID_ARG
    # value asymmetry
    with pytest.raises(B.AmgError) as e:
        B.amg_setup(*csr_dev(rp, np.array([0, 1, 0, 1], np.int32), np.array([2.0, -1.0, -0.5, 2.0])), dev(np.ones(2)))
    assert e.value.status == B.AMG_ERR_INVALID_ARG
    # parameters out of range
    mat = P.poisson2d(4)
    for bad in (dict(coupled_post=2), dict(coupled_post=-2), dict(pre_sweeps=-1), dict(sweeps_per_level=0)):
        with pytest.raises(B.AmgError) as e:
            B.amg_setup(*csr_dev(*mat), dev(np.ones(16)), B.amg_default_params(**bad))
        assert e.value.status == B.AMG_ERR_INVALID_ARG
    # an aggregate with three members
    with pytest.raises(B.AmgError) as e:
        mat = P.poisson2d(4)
        B.cwm_galerkin(*csr_dev(*mat), 14, dev(np.array([0, 0, 0] + list(range(1, 14)), np.int32)), dev(np.ones(16)))
    assert e.value.status == B.AMG_ERR_INVALID_ARG


def test_loop_cap_reports_timeout():
    """A cap of one iteration per proposal chain cannot finish the Suitor rounds: the kernel
    gives up, reports AMG_ERR_TIMEOUT and leaves the context usable."""
    mat = P.poisson2d(32)
    with pytest.raises(B.AmgError) as e:
        B.amg_setup(*csr_dev(*mat), dev(np.ones(1024)), B.amg_default_params(loop_cap=1))
    assert e.value.status == B.AMG_ERR_TIMEOUT
    h = B.amg_setup(*csr_dev(*mat), dev(np.ones(1024)))
    assert B.amg_num_levels(h) > 1
    h.free()


def test_setup_deterministic():
    mat = P.lognormal_diffusion(16, seed=4)
    n = len(mat[0]) - 1
    outs = []
    for _ in range(2):
        h = B.amg_setup(*csr_dev(*mat), dev(np.ones(n)), B.amg_default_params(sweeps_per_level=3, coarse_max=50))
        lv = [B.amg_level_export(h, k) for k in range(B.amg_num_levels(h))]
        outs.append([(host(L["ci"]), host(L["val"])) for L in lv])
        h.free()
    assert len(outs[0]) == len(outs[1])
    for (c1, v1), (c2, v2) in zip(*outs):
        assert np.array_equal(c1, c2) and bits_equal(v1, v2)


def test_vcycle_barrier_wait_reports_timeout():
    """The fused V-cycle tail waits at grid barriers with a bounded poll count.  With a
    cap of one poll the waits give up: amg_vcycle reports AMG_ERR_TIMEOUT, and the
    context stays usable for a normal hierarchy afterwards."""
    n = 100
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    val = np.full(n, 2.0)
    h = B.amg_setup(*csr_dev(rp, ci, val), dev(np.ones(n)),
                    B.amg_default_params(loop_cap=1, coarse_max=0, tail_rows=0))
    try:
        w = torch.empty(n, dtype=torch.float64, device="cuda")
        with pytest.raises(B.AmgError) as e:
            B.amg_vcycle(h, dev(np.ones(n)), w)
        assert e.value.status == B.AMG_ERR_TIMEOUT
    finally:
        h.free()
    mat = P.poisson2d(16)
    h = B.amg_setup(*csr_dev(*mat), dev(np.ones(256)))
    x = torch.zeros(256, dtype=torch.float64, device="cuda")
    st, info = B.amg_pcg_solve(h, dev(np.ones(256)), x)
    assert st == B.AMG_OK
    h.free()


def test_paper_coarse_size_matches_oracle():
    """coarse_max = -1 (the paper's floor(40 n^(1/3))): the same levels as the oracle."""
    mat = P.poisson3d(32)
    n = len(mat[0]) - 1
    H = oracle.Hierarchy(*mat, np.ones(n), sweeps=3, coarse_max=-1)
    h = B.amg_setup(*csr_dev(*mat), dev(np.ones(n)), B.amg_default_params(sweeps_per_level=3, coarse_max=-1))
    try:
        assert B.amg_num_levels(h) == H.nl == 3
        for k in range(H.nl):
            got, ref = B.amg_level_export(h, k), H.level(k)
            assert np.array_equal(host(got["ci"]), ref["ci"]) and bits_equal(host(got["val"]), ref["val"])
    finally:
        h.free()

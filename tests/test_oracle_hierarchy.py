"""Pins of the oracle's aggregation (Algorithm 2), prolongator (Sec. 2.2), Galerkin
product (Sec. 2.1) and multi-sweep hierarchy (Sec. 5) against library products,
closed forms and invariants (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1810_04221_gb300 import problems as P


def _P_matrix(agg, p, nc):
    n = len(agg)
    return sp.csr_matrix((p, (np.arange(n), agg)), shape=(n, nc))


def _one_sweep(rp, ci, val, v):
    w = oracle.edge_weights(rp, ci, val, v)
    mate = oracle.greedy_match(rp, ci, w)
    agg, nc, npairs, nsing = oracle.aggregate(mate)
    p, vc = oracle.prolongator(agg, nc, v)
    return mate, agg, nc, npairs, nsing, p, vc


# ------------------------------------------------------------ aggregation ----

@pytest.mark.parametrize("seed", range(4))
def test_aggregation_counts_and_order(seed):
    rp, ci, val = P.random_spd(3000, 6.0, seed=seed, ties=seed % 2 == 1)
    v = np.random.default_rng(seed).uniform(0.5, 2, 3000)
    mate, agg, nc, npairs, nsing, p, vc = _one_sweep(rp, ci, val, v)
    assert nc == npairs + nsing
    assert npairs == int(np.sum(mate >= 0)) // 2
    # every aggregate is a matched pair or a singleton
    members = [[] for _ in range(nc)]
    for i, a in enumerate(agg):
        members[a].append(i)
    for I, m in enumerate(members):
        assert len(m) in (1, 2)
        if len(m) == 2:
            assert mate[m[0]] == m[1]
        else:
            assert mate[m[0]] < 0
    # ids follow the smallest member (U scanned in ascending order)
    firsts = [m[0] for m in members]
    assert firsts == sorted(firsts)


def test_aggregation_no_edges():
    mate = -np.ones(7, np.int32)
    agg, nc, npairs, nsing = oracle.aggregate(mate)
    assert nc == 7 and npairs == 0 and nsing == 7 and np.array_equal(agg, np.arange(7))


# ------------------------------------------------------------ prolongator ----

@pytest.mark.parametrize("seed", range(3))
def test_prolongator_orthonormal_and_reproduces_v(seed):
    rp, ci, val = P.random_spd(2000, 5.0, seed=seed)
    v = np.random.default_rng(seed).uniform(-2, 2, 2000)
    v[::97] = 0.0  # zero entries exercise the singleton special case
    mate, agg, nc, _, _, p, vc = _one_sweep(rp, ci, val, v)
    Pm = _P_matrix(agg, p, nc)
    PtP = (Pm.T @ Pm).toarray()
    assert np.abs(PtP - np.eye(nc)).max() < 1e-15 * 4
    assert np.abs(Pm @ vc - v).max() <= 1e-15 * np.abs(v).max() * 4
    assert np.abs(Pm.T @ v - vc).max() <= 1e-15 * np.abs(v).max() * 4


# -------------------------------------------------------------- Galerkin ----

@pytest.mark.parametrize("kind,seed", [("rand", 0), ("rand", 1), ("ties", 2), ("diff", 3), ("zeros", 4)])
def test_galerkin_vs_dense_product(kind, seed):
    if kind == "diff":
        rp, ci, val = P.lognormal_diffusion(10, seed=seed)
        n = len(rp) - 1
        v = np.ones(n)
    else:
        n = 1500
        rp, ci, val = P.random_spd(n, 6.0, seed=seed, ties=kind == "ties",
                                   explicit_zeros=0.2 if kind == "zeros" else 0.0)
        v = np.random.default_rng(seed).uniform(0.5, 2, n)
    mate, agg, nc, _, _, p, vc = _one_sweep(rp, ci, val, v)
    rpc, cic, valc = oracle.galerkin(rp, ci, val, agg, nc, p)
    assert oracle.check_csr(rpc, cic)
    A = P.to_scipy(rp, ci, val)
    Pm = _P_matrix(agg, p, nc)
    dense = (Pm.T @ A @ Pm).toarray()
    got = sp.csr_matrix((valc, cic, rpc), shape=(nc, nc)).toarray()
    scale = np.abs(val).max()
    assert np.abs(got - dense).max() <= 1e-14 * scale
    # pattern = every (I, J) hit by a stored fine entry (structural zeros kept)
    pat = sp.csr_matrix((np.ones_like(val), ci, rp), shape=(n, n))
    B = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, nc))
    hit = (B.T @ pat @ B).tocsr()
    hit.sort_indices()
    assert np.array_equal(hit.indptr, rpc) and np.array_equal(hit.indices, cic)
    # bit symmetry of A_c and A_c v_c = P^T (A v)
    assert oracle.check_symmetric(rpc, cic, valc)
    Ac = sp.csr_matrix((valc, cic, rpc), shape=(nc, nc))
    lhs, rhs = Ac @ vc, Pm.T @ (A @ v)
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(rhs).max()


def test_galerkin_spd_by_cholesky():
    rp, ci, val = P.random_spd(800, 6.0, seed=11)
    v = np.ones(800)
    mate, agg, nc, _, _, p, vc = _one_sweep(rp, ci, val, v)
    rpc, cic, valc = oracle.galerkin(rp, ci, val, agg, nc, p)
    Ac = sp.csr_matrix((valc, cic, rpc), shape=(nc, nc)).toarray()
    np.linalg.cholesky(Ac)  # raises if not s.p.d.


def test_galerkin_binary_p_row_sums():
    # with a binary P (p = 1) the coarse row sums equal P^T (A 1): A_c 1 = P^T A 1
    rp, ci, val = P.random_spd(1000, 5.0, seed=5)
    mate, agg, nc, _, _, _, _ = _one_sweep(rp, ci, val, np.ones(1000))
    ones = np.ones(1000)
    rpc, cic, valc = oracle.galerkin(rp, ci, val, agg, nc, ones)
    Ac = sp.csr_matrix((valc, cic, rpc), shape=(nc, nc))
    Bm = _P_matrix(agg, ones, nc)
    lhs = Ac @ np.ones(nc)
    rhs = Bm.T @ (P.to_scipy(rp, ci, val) @ ones)
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(rhs).max()


# ------------------------------------------------------------- hierarchy ----

def test_hierarchy_poisson2d_closed_form():
    """64^2 Poisson, v = 1, 2 sweeps per level: 2x2 blocks on every level,
    A^k = 2^{-k} L_5 on (64/2^k)^2, v_k = 2^k, n = 4096, 1024, 256, 64, 16."""
    rp, ci, val = P.poisson2d(64)
    H = oracle.Hierarchy(rp, ci, val, np.ones(4096), sweeps=2, coarse_max=40)
    assert H.nl == 5
    ns = [H.level_n(k) for k in range(5)]
    zs = [H.level_nnz(k) for k in range(5)]
    assert ns == [4096, 1024, 256, 64, 16]
    assert zs == [5 * m * m - 4 * m for m in (64, 32, 16, 8, 4)]
    vc, cr = H.stats()
    assert abs(vc - (20224 + 4992 + 1216 + 288 + 64) / 20224) < 1e-15
    assert abs(cr - 16.0 / 5.0) < 1e-15  # (1/nl) * 4 ratios of 4
    for k in range(1, 5):
        L = H.level(k)
        m = 64 >> k
        ref = P.to_scipy(*P.poisson2d(m)) * (0.5 ** k)
        got = P.to_scipy(L["rp"], L["ci"], L["val"])
        assert abs(got - ref).max() < 1e-14
        assert np.abs(L["v"] - 2.0 ** k).max() < 1e-14
    # level-0 aggregates are 2x2 blocks with P entries 1/2
    L0 = H.level(0)
    y, x = np.divmod(np.arange(4096), 64)
    assert np.array_equal(L0["agg"], (y // 2) * 32 + x // 2)
    assert np.abs(L0["p"] - 0.5).max() < 1e-15
    # sweep 1 = x-pairs, sweep 2 = y-pairs of the 32x64 intermediate grid
    assert np.array_equal(H.sweep_mate(0, 0), np.arange(4096) ^ 1)
    yy, xx = np.divmod(np.arange(2048), 32)
    assert np.array_equal(H.sweep_mate(0, 1), (yy ^ 1) * 32 + xx)


def test_hierarchy_poisson3d_closed_form():
    """m^3 Poisson, v = 1, 3 sweeps: x-, y-, z-pairs -> 2x2x2 cubes, A_c = L_7 / 2,
    v_c = 2 sqrt 2; the coarse level has the same weights (7/6), so it repeats."""
    m = 16
    rp, ci, val = P.poisson3d(m)
    H = oracle.Hierarchy(rp, ci, val, np.ones(m ** 3), sweeps=3, coarse_max=10)
    assert [H.level_n(k) for k in range(H.nl)] == [4096, 512, 64, 8]
    for k in range(1, H.nl):
        L = H.level(k)
        mk = m >> k
        ref = P.to_scipy(*P.poisson3d(mk)) * (0.5 ** k)
        assert abs(P.to_scipy(L["rp"], L["ci"], L["val"]) - ref).max() < 1e-14
        assert np.abs(L["v"] - 8.0 ** (k / 2)).max() < 1e-13
    z, r = np.divmod(np.arange(m ** 3), m * m)
    y, x = np.divmod(r, m)
    h = m // 2
    assert np.array_equal(H.level(0)["agg"], ((z // 2) * h + y // 2) * h + x // 2)
    assert np.array_equal(H.sweep_mate(0, 0), np.arange(m ** 3) ^ 1)


@pytest.mark.parametrize("sweeps", [1, 2, 3])
def test_hierarchy_composed_prolongator(sweeps):
    """A^{k+1} = (P_1...P_S)^T A^k (P_1...P_S) up to rounding; P^k orthonormal; P^k v_{k+1} = v_k."""
    rp, ci, val = P.lognormal_diffusion(12, seed=1)
    n = len(rp) - 1
    H = oracle.Hierarchy(rp, ci, val, np.ones(n), sweeps=sweeps, coarse_max=50)
    assert H.nl >= 2
    for k in range(H.nl - 1):
        F, Cl = H.level(k), H.level(k + 1)
        Pm = _P_matrix(F["agg"], F["p"], Cl["n"])
        A = P.to_scipy(F["rp"], F["ci"], F["val"])
        dense = (Pm.T @ A @ Pm).toarray()
        got = P.to_scipy(Cl["rp"], Cl["ci"], Cl["val"]).toarray()
        assert np.abs(got - dense).max() <= 1e-13 * np.abs(dense).max()
        assert np.abs((Pm.T @ Pm).toarray() - np.eye(Cl["n"])).max() < 1e-14
        assert np.abs(Pm @ Cl["v"] - F["v"]).max() < 1e-13 * np.abs(F["v"]).max()
        assert np.bincount(F["agg"]).max() <= 2 ** sweeps
        assert oracle.check_symmetric(Cl["rp"], Cl["ci"], Cl["val"])
        # l1 row norms
        assert np.array_equal(F["dl1"], np.asarray(abs(A).sum(axis=1)).ravel()) or \
            np.abs(F["dl1"] - np.asarray(abs(A).sum(axis=1)).ravel()).max() < 1e-13 * F["dl1"].max()


def test_paper_coarse_size():
    """The paper's coarse size floor(40 n^(1/3)) (Sec. 5): exactly 40 k for n = k^3, and the
    defining bounds m^3 <= 64000 n < (m + 1)^3 elsewhere."""
    for k in (1, 2, 16, 100, 128, 160):
        assert oracle.paper_coarse_max(k ** 3) == 40 * k
    for n in (2, 3, 999, 1001, 4095, 4097, 786432, 884736, 4096000 - 1, 2 ** 31 - 1):
        m = oracle.paper_coarse_max(n)
        assert m ** 3 <= 64000 * n < (m + 1) ** 3, n


def test_hierarchy_paper_coarse_size():
    """coarse_max = -1 stops where the paper's rule does: 3D Poisson 32^3 (n = 32768, coarse
    size 1280) keeps the 4096-row level (> 1280) and stops at 512 rows."""
    rp, ci, val = P.poisson3d(32)
    H = oracle.Hierarchy(rp, ci, val, np.ones(32 ** 3), sweeps=3, coarse_max=-1)
    assert [H.level_n(k) for k in range(H.nl)] == [32768, 4096, 512]
    H2 = oracle.Hierarchy(rp, ci, val, np.ones(32 ** 3), sweeps=3, coarse_max=4096)
    assert H2.nl == 2


def test_hierarchy_stops_without_pairs():
    # diagonal matrix: no edge, so no coarse level is made
    n = 50
    rp = np.arange(n + 1, dtype=np.int32)
    H = oracle.Hierarchy(rp, np.arange(n, dtype=np.int32), np.full(n, 3.0), np.ones(n),
                         sweeps=2, coarse_max=4)
    assert H.nl == 1


def test_hierarchy_rejects_bad_input():
    rp = np.array([0, 2, 4], np.int32)
    with pytest.raises(ValueError):
        oracle.Hierarchy(rp, np.array([1, 0, 0, 1], np.int32), np.ones(4), np.ones(2), coarse_max=1)
    with pytest.raises(ValueError):  # zero diagonal
        oracle.Hierarchy(rp, np.array([0, 1, 0, 1], np.int32), np.array([0.0, -1, -1, 2]),
                         np.ones(2), coarse_max=1)


def test_hierarchy_stall_ratio_stops_hub_growth():
    """With strongly heterogeneous coefficients one aggregate can become a hub that all
    remaining vertices touch (a star): each sweep then pairs one vertex.  The optional
    stall ratio stops after the first level that coarsens by less than the ratio."""
    mat = P.lognormal_diffusion(24, seed=0)
    n = len(mat[0]) - 1
    H = oracle.Hierarchy(*mat, np.ones(n), sweeps=3, coarse_max=10, max_levels=40)
    ns = [H.level_n(k) for k in range(H.nl)]
    H2 = oracle.Hierarchy(*mat, np.ones(n), sweeps=3, coarse_max=10, max_levels=40, stall_ratio=1.2)
    ns2 = [H2.level_n(k) for k in range(H2.nl)]
    k = next(i for i in range(1, len(ns)) if ns[i - 1] < 1.2 * ns[i])
    assert ns2 == ns[:k + 1]


# ------------------------------------------------ binary32 Galerkin variant ----

def test_galerkin_fp32_accumulates_in_binary32():
    """Hand-worked case: one aggregate {0, 1}, p = 1, a_00 = 1, a_01 = a_10 = 2^-24,
    a_11 = 1/2.  The four terms in canonical order are 1, 2^-24, 2^-24, 1/2.  In binary32
    1 + 2^-24 rounds (to even) back to 1 twice, so the entry is exactly 1.5; a double sum
    rounded once at the end would give 1.5 + 2^-23 instead."""
    rp = np.array([0, 2, 4], np.int32)
    ci = np.array([0, 1, 0, 1], np.int32)
    val = np.array([1.0, 2.0 ** -24, 2.0 ** -24, 0.5])
    agg = np.zeros(2, np.int32)
    rpc, cic, valc = oracle.galerkin(rp, ci, val, agg, 1, np.ones(2), fp32=True)
    assert valc[0] == 1.5
    rpc, cic, valc = oracle.galerkin(rp, ci, val, agg, 1, np.ones(2))
    assert valc[0] == 1.5 + 2.0 ** -23


def test_galerkin_fp32_rounds_the_inputs():
    """p = 1 + 2^-30 is 1 in binary32, so the binary32 entry of a singleton aggregate is
    exactly float(a_00); the binary64 entry carries the factor (1 + 2^-30)^2."""
    rp = np.array([0, 1], np.int32)
    ci = np.array([0], np.int32)
    val = np.array([3.0])
    p = np.array([1.0 + 2.0 ** -30])
    assert oracle.galerkin(rp, ci, val, np.zeros(1, np.int32), 1, p, fp32=True)[2][0] == 3.0
    assert oracle.galerkin(rp, ci, val, np.zeros(1, np.int32), 1, p)[2][0] == (p[0] * p[0]) * 3.0


@pytest.mark.parametrize("kind,seed", [("rand", 0), ("ties", 2), ("diff", 3)])
def test_galerkin_fp32_error_bound(kind, seed):
    """Each binary32 entry is within 9u (u = 2^-24) of the exact P^T A P entry, relative to
    (|P|^T |A| |P|)_IJ: three input roundings and two products per term, at most three
    additions over at most four terms.  Entries are binary32 numbers, the pattern is the
    binary64 product's, and A_c is bit-symmetric."""
    if kind == "diff":
        rp, ci, val = P.lognormal_diffusion(10, seed=seed)
        n = len(rp) - 1
        v = np.ones(n)
    else:
        n = 1500
        rp, ci, val = P.random_spd(n, 6.0, seed=seed, ties=kind == "ties")
        v = np.random.default_rng(seed).uniform(0.5, 2, n)
    mate, agg, nc, _, _, p, vc = _one_sweep(rp, ci, val, v)
    r32, c32, v32 = oracle.galerkin(rp, ci, val, agg, nc, p, fp32=True)
    r64, c64, v64 = oracle.galerkin(rp, ci, val, agg, nc, p)
    assert np.array_equal(r32, r64) and np.array_equal(c32, c64)
    assert np.array_equal(v32, v32.astype(np.float32).astype(np.float64))
    assert oracle.check_symmetric(r32, c32, v32)
    A = P.to_scipy(rp, ci, val)
    Pm = _P_matrix(agg, p, nc)
    exact = (Pm.T @ A @ Pm).toarray()
    mag = (abs(Pm).T @ abs(A) @ abs(Pm)).toarray()
    got = sp.csr_matrix((v32, c32, r32), shape=(nc, nc)).toarray()
    assert np.all(np.abs(got - exact) <= 9 * 2.0 ** -24 * mag + 1e-300)
    # and it is not the binary64 product: some entry differs
    assert np.any(v32 != v64)


def test_hierarchy_fp32_galerkin_poisson_closed_form():
    """3D Poisson, v = 1: equal entries see equal binary32 roundings, so ties stay ties and
    the hierarchy keeps the closed-form structure (2x2x2 cubes, A^k = 2^-k L_7 on
    (16/2^k)^3); the values carry only the binary32 rounding of the p's (1/sqrt 2 is not a
    binary32 number) and of three products per level: within 3 * 9u per level relative."""
    rp, ci, val = P.poisson3d(16)
    n = len(rp) - 1
    H64 = oracle.Hierarchy(rp, ci, val, np.ones(n), sweeps=3, coarse_max=10)
    H32 = oracle.Hierarchy(rp, ci, val, np.ones(n), sweeps=3, coarse_max=10, galerkin_fp32_from=1)
    assert H32.nl == H64.nl == 4
    for k in range(H64.nl):
        a, b = H64.level(k), H32.level(k)
        assert np.array_equal(a["rp"], b["rp"]) and np.array_equal(a["ci"], b["ci"])
        if k < H64.nl - 1:
            assert np.array_equal(a["agg"], b["agg"])
        m = 16 >> k
        rows = np.repeat(np.arange(m ** 3), np.diff(b["rp"]))
        ref = np.where(b["ci"] == rows, 6.0, -1.0) * 0.5 ** k
        assert np.all(np.abs(b["val"] - ref) <= k * 27 * 2.0 ** -24 * np.abs(ref))
        if k >= 1:
            assert np.any(b["val"] != ref)


def test_hierarchy_fp32_galerkin_from_level():
    """galerkin_fp32_from = 2 keeps levels 0 and 1 binary64 (bit-equal to the plain
    hierarchy) and forms the later levels in binary32."""
    rp, ci, val = P.lognormal_diffusion(12, seed=5)
    n = len(rp) - 1
    H64 = oracle.Hierarchy(rp, ci, val, np.ones(n), sweeps=2, coarse_max=20)
    H2 = oracle.Hierarchy(rp, ci, val, np.ones(n), sweeps=2, coarse_max=20, galerkin_fp32_from=2)
    assert H64.nl >= 4
    for k in (0, 1):
        assert np.array_equal(H64.level(k)["val"], H2.level(k)["val"])
    L2 = H2.level(2)["val"]
    assert np.array_equal(L2, L2.astype(np.float32).astype(np.float64))

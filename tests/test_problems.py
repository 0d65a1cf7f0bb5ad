"""Pins of the seeded input generators (the synthetic stand-ins for the paper's scalar
diffusion and linear elasticity workloads, Sec. 5) against their stated recipes: brute
force on tiny grids, closed forms, and the physics that fixes them (rigid-body modes)."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1810_04221_gb300 import problems as P


def _dense(mat):
    rp, ci, val = mat
    n = len(rp) - 1
    return sp.csr_matrix((val, ci, rp), shape=(n, n)).toarray()


def test_diffusion_fv_brute_force():
    """Interior faces: T = 2 k1 k2 / (k1 + k2); every domain face: Dirichlet through the
    half-cell transmissibility 2 k; A = sum over faces of T (e_i - e_j)(e_i - e_j)^T plus
    the boundary terms, built here cell by cell."""
    rng = np.random.default_rng(0)
    shape = (2, 3, 4)  # (z, y, x)
    kappa = np.exp(rng.standard_normal(shape))
    A = _dense(P.diffusion_fv(kappa))
    mz, my, mx = shape
    cell = lambda z, y, x: (z * my + y) * mx + x  # noqa: E731
    ref = np.zeros((mz * my * mx,) * 2)
    for z, y, x in itertools.product(range(mz), range(my), range(mx)):
        i = cell(z, y, x)
        for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            zz, yy, xx = z + dz, y + dy, x + dx
            if 0 <= zz < mz and 0 <= yy < my and 0 <= xx < mx:
                k1, k2 = kappa[z, y, x], kappa[zz, yy, xx]
                t = 2 * k1 * k2 / (k1 + k2)
                ref[i, i] += t
                ref[i, cell(zz, yy, xx)] -= t
            else:
                ref[i, i] += 2 * kappa[z, y, x]
    assert np.allclose(A, ref, rtol=1e-14, atol=0)
    assert np.array_equal(A, A.T)  # bit-symmetric
    np.linalg.cholesky(A)


def test_diffusion_fv_constant_kappa_closed_form():
    """kappa = 1: off-diagonals -1, diagonal 6 plus one per domain face of the cell."""
    m = 5
    A = _dense(P.diffusion_fv(np.ones((m, m, m))))
    z, y, x = np.meshgrid(*(np.arange(m),) * 3, indexing="ij")
    faces = sum(((c == 0).astype(int) + (c == m - 1).astype(int)) for c in (z, y, x)).ravel()
    assert np.array_equal(np.diag(A), 6.0 + faces)
    off = A - np.diag(np.diag(A))
    assert set(np.unique(off)) <= {-1.0, 0.0}
    assert np.array_equal((off != 0).sum(axis=1), 6 - faces)


def test_lognormal_kappa_distribution():
    k = P.lognormal_kappa(40, sigma=2.0, seed=1)
    lk = np.log(k).ravel()
    assert abs(lk.mean()) < 0.05 and abs(lk.std() - 2.0) < 0.05
    assert np.array_equal(k, P.lognormal_kappa(40, sigma=2.0, seed=1))  # seeded


def _rigid_modes(h):
    """Translations and linearised rotations of the 8 nodes of a cube of side h."""
    off = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float) * h
    modes = []
    for c in range(3):
        u = np.zeros((8, 3))
        u[:, c] = 1.0
        modes.append(u.ravel())
    for axis in range(3):
        w = np.zeros(3)
        w[axis] = 1.0
        modes.append(np.cross(w, off).ravel())
    return np.array(modes).T  # 24 x 6


def test_q1_element_stiffness_rigid_body_modes():
    """The element stiffness is symmetric positive semidefinite, annihilates the six rigid
    motions and nothing else (2x2x2 Gauss integrates the Q1 stiffness exactly)."""
    h = 0.25
    K = P._q1_element_stiffness(h, 1.0, 0.3)
    assert np.array_equal(K, K.T)
    R = _rigid_modes(h)
    assert np.abs(K @ R).max() <= 1e-13 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert (np.abs(ev[:6]) <= 1e-13 * ev[-1]).all() and ev[6] > 1e-3 * ev[-1]


def _nb(m):
    """Ordered pairs (i, j) with |i - j| <= 1 among m consecutive grid positions."""
    return m + 2 * (m - 1)


@pytest.mark.parametrize("nodes", [4, 6])
def test_elasticity_q1_sizes_and_spd(nodes):
    """x = 0 face clamped by elimination: n = 3 (nodes - 1) nodes^2; exactly 9 entries per
    ordered pair of free nodes sharing an element (the assembled pattern, stored zeros
    included); symmetric positive definite."""
    mat = P.elasticity_q1(nodes)
    n = len(mat[0]) - 1
    assert n == 3 * (nodes - 1) * nodes * nodes
    assert len(mat[1]) == 9 * _nb(nodes - 1) * _nb(nodes) ** 2
    A = _dense(mat)
    assert np.array_equal(A, A.T)
    np.linalg.cholesky(A)
    assert (np.diag(A) > 0).all()
    rp, ci, _ = mat
    assert all((np.diff(ci[rp[i]:rp[i + 1]]) > 0).all() for i in range(n))


def test_elasticity_q1_brute_force_assembly():
    """Element by element: A = sum over the (nodes-1)^3 cubes of the 24x24 element stiffness
    on the cube's dofs, clamped rows and columns removed; the stored pattern is every pair
    of dofs of nodes within one grid step in each direction, and stored zeros occur exactly
    where the assembled sum cancels."""
    nodes = 4
    rp, ci, val = P.elasticity_q1(nodes)
    ne, h = nodes - 1, 1.0 / (nodes - 1)
    Ke = P._q1_element_stiffness(h, 1.0, 0.3)
    full = np.zeros((3 * nodes ** 3,) * 2)
    coupled = np.zeros_like(full, dtype=bool)
    for ez, ey, ex in itertools.product(range(ne), repeat=3):
        nd = [((ez + (a >> 2 & 1)) * nodes + ey + (a >> 1 & 1)) * nodes + ex + (a & 1) for a in range(8)]
        dofs = np.array([3 * q + c for q in nd for c in range(3)])
        full[np.ix_(dofs, dofs)] += Ke
        coupled[np.ix_(dofs, dofs)] = True
    free = np.array([d for d in range(3 * nodes ** 3) if (d // 3) % nodes != 0])
    ref, pat = full[np.ix_(free, free)], coupled[np.ix_(free, free)]
    n = len(free)
    A = _dense((rp, ci, val))
    S = np.zeros((n, n), bool)
    S[np.repeat(np.arange(n), np.diff(rp)), ci] = True
    assert np.array_equal(S, pat)
    assert np.abs(A - ref).max() <= 1e-14 * np.abs(ref).max()
    zeros = S & (A == 0)
    assert zeros.sum() > 0 and (np.abs(ref[zeros]) <= 1e-14 * np.abs(ref).max()).all()


def test_elasticity_q1_full_size_counts():
    """64^3 nodes, x = 0 clamped: n = 3 * 63 * 64^2 = 774,144 and nnz = 9 * 187 * 190^2 =
    60,756,300 by the pair count above (both without building the matrix)."""
    assert 3 * 63 * 64 * 64 == 774144
    assert 9 * _nb(63) * _nb(64) ** 2 == 60756300


def test_random_block3_spd_pattern():
    """Block rows 3b..3b+2 share their columns, in aligned triples; hub block rows far longer
    than the mean; stored zeros inside blocks; bit-symmetric and s.p.d."""
    rp, ci, val = P.random_block3_spd(300, avg_blocks=5.0, n_hubs=2, hub_blocks=60, seed=3)
    n = len(rp) - 1
    assert n == 900
    lens = np.diff(rp)
    for b in range(n // 3):
        r = [ci[rp[3 * b + i]:rp[3 * b + i + 1]] for i in range(3)]
        assert np.array_equal(r[0], r[1]) and np.array_equal(r[0], r[2])
        assert len(r[0]) % 3 == 0 and (r[0][0::3] % 3 == 0).all()
        assert np.array_equal(r[0][1::3], r[0][0::3] + 1) and np.array_equal(r[0][2::3], r[0][0::3] + 2)
    assert lens.max() >= 3 * 60 and lens.mean() < 3 * 10
    assert (val == 0).sum() > 0
    A = _dense((rp, ci, val))
    assert np.array_equal(A, A.T)
    np.linalg.cholesky(A)

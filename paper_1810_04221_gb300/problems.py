"""Seeded synthetic s.p.d. test matrices shaped like the paper's workloads.

The paper's own matrices (anisotropic FEM, Lame elasticity, Parflow Darcy) are not
available, so these generators stand in for them: scalar Poisson stencils, a
cell-centred finite-volume diffusion operator with a lognormal coefficient (Parflow-like),
a trilinear Q1 elasticity operator (vector PDE), and random s.p.d. graphs for edge cases.

This module is input generation only: it holds none of the coarsening arithmetic, and it
is the one module both the CUDA path's tests/bench and the CPU oracle's tests read.
Every matrix is returned as (row_ptr int32[n+1], col int32[nnz], val float64[nnz]) with
strictly ascending columns in every row and bit-symmetric values.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _to_csr(mat: sp.spmatrix):
    m = sp.csr_matrix(mat)
    m.sum_duplicates()
    m.sort_indices()
    return (m.indptr.astype(np.int32), m.indices.astype(np.int32), m.data.astype(np.float64))


def _lap1d(m: int) -> sp.csr_matrix:
    return sp.diags([-np.ones(m - 1), 2.0 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1], format="csr")


def poisson2d(m: int):
    """5-point Laplacian on an m x m interior grid, Dirichlet rows eliminated.

    diag 4, off-diagonal -1, vertex index y*m + x; n = m^2, nnz = 5m^2 - 4m.
    """
    eye = sp.identity(m, format="csr")
    t = _lap1d(m)
    return _to_csr(sp.kron(eye, t) + sp.kron(t, eye))


def poisson3d(m: int):
    """7-point Laplacian on an m^3 interior grid, Dirichlet rows eliminated.

    diag 6, off-diagonal -1, vertex index (z*m + y)*m + x; nnz = 7m^3 - 6m^2.
    """
    eye = sp.identity(m, format="csr")
    t = _lap1d(m)
    a = sp.kron(sp.kron(eye, eye), t) + sp.kron(sp.kron(eye, t), eye) + sp.kron(sp.kron(t, eye), eye)
    return _to_csr(a)


def lognormal_kappa(m: int, sigma: float = 2.0, seed: int = 0) -> np.ndarray:
    """Per-cell permeability kappa = exp(N(0, sigma^2)), i.i.d., shape (m, m, m) as [z, y, x]."""
    rng = np.random.default_rng(seed)
    return np.exp(sigma * rng.standard_normal((m, m, m)))


def diffusion_fv(kappa: np.ndarray):
    """Cell-centred FV operator of -div(kappa grad u) on the unit-spacing grid of `kappa`.

    Interior face transmissibility is the harmonic mean 2 k1 k2 / (k1 + k2); every domain
    face carries a Dirichlet condition u = 0 through the half-cell transmissibility
    2 k_cell (a no-flow boundary would make A singular).  Each face value is computed once
    and used for both (i, j) and (j, i), so A is bit-symmetric.
    """
    mz, my, mx = kappa.shape
    n = mz * my * mx
    idx = np.arange(n, dtype=np.int64).reshape(mz, my, mx)
    diag = np.zeros((mz, my, mx))
    rows, cols, vals = [], [], []
    for axis in (2, 1, 0):  # x, y, z
        k0 = np.moveaxis(kappa, axis, 0)
        i0 = np.moveaxis(idx, axis, 0)
        d0 = np.moveaxis(diag, axis, 0)  # a view into diag
        t = 2.0 * k0[:-1] * k0[1:] / (k0[:-1] + k0[1:])
        d0[:-1] += t
        d0[1:] += t
        d0[0] += 2.0 * k0[0]
        d0[-1] += 2.0 * k0[-1]
        a, b = i0[:-1].ravel(), i0[1:].ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [-t.ravel(), -t.ravel()]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    mat = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                        shape=(n, n))
    return _to_csr(mat)


def lognormal_diffusion(m: int, sigma: float = 2.0, seed: int = 0):
    """Parflow-like heterogeneous diffusion on m^3 cells (log-kappa ~ N(0, sigma^2))."""
    return diffusion_fv(lognormal_kappa(m, sigma, seed))


def _q1_element_stiffness(h: float, E: float, nu: float) -> np.ndarray:
    """24x24 stiffness of a cube element of side h, 2x2x2 Gauss, dof order node*3 + comp.

    Local node a has offsets (ax, ay, az) = (a & 1, (a >> 1) & 1, (a >> 2) & 1).
    """
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    g = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    off = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=float)
    K = np.zeros((24, 24))
    for gx in g:
        for gy in g:
            for gz in g:
                xi = np.array([gx, gy, gz])
                s = 2 * off - 1  # node sign per direction
                # dN/dxi for trilinear N_a = prod (1 + s_a xi)/2
                f = (1 + s * xi) / 2
                dN = np.empty((8, 3))
                dN[:, 0] = s[:, 0] / 2 * f[:, 1] * f[:, 2]
                dN[:, 1] = f[:, 0] * s[:, 1] / 2 * f[:, 2]
                dN[:, 2] = f[:, 0] * f[:, 1] * s[:, 2] / 2
                dNdx = dN * (2.0 / h)
                B = np.zeros((6, 24))
                for a in range(8):
                    bx, by, bz = dNdx[a]
                    B[0, 3 * a], B[1, 3 * a + 1], B[2, 3 * a + 2] = bx, by, bz
                    B[3, 3 * a], B[3, 3 * a + 1] = by, bx
                    B[4, 3 * a + 1], B[4, 3 * a + 2] = bz, by
                    B[5, 3 * a], B[5, 3 * a + 2] = bz, bx
                K += B.T @ D @ B * (h / 2) ** 3
    return 0.5 * (K + K.T)


def elasticity_q1(nodes: int = 64, E: float = 1.0, nu: float = 0.3):
    """Trilinear Q1 linear elasticity on the unit cube with nodes^3 nodes, face x=0 clamped.

    The clamped dofs are eliminated (not kept as identity rows).  Unknowns are
    dof-interleaved: 3 * node + component over the free nodes in (z, y, x) order.

    The stored pattern is the assembled one: every (dof, dof) pair of two nodes that share
    an element, 9 entries per such node pair (27 node neighbours inside the grid), whether
    or not the assembled sum is exactly zero.  With nodes = 64 that is n = 774,144 and
    nnz = 9 * 187 * 190^2 = 60,756,300 (about 78.5 per row); some 11.5M of them are exact
    zeros of the assembly (couplings that cancel between the elements around an edge or a
    face), kept as stored zeros.  The nonzero values are the element sums, made exactly
    symmetric as 0.5 (K + K^T).
    """
    ne = nodes - 1
    h = 1.0 / ne
    Ke = _q1_element_stiffness(h, E, nu)
    ez, ey, ex = np.meshgrid(np.arange(ne), np.arange(ne), np.arange(ne), indexing="ij")
    base = ((ez * nodes + ey) * nodes + ex).ravel().astype(np.int64)
    loc = np.array([(a & 1) + ((a >> 1) & 1) * nodes + ((a >> 2) & 1) * nodes * nodes
                    for a in range(8)], dtype=np.int64)
    enodes = base[:, None] + loc[None, :]                              # (nel, 8)
    edofs = (3 * enodes[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 24)
    ndof = 3 * nodes ** 3
    # free-dof numbering: drop nodes with x == 0
    node_x = np.arange(nodes ** 3) % nodes
    free_node = node_x != 0
    new_node = -np.ones(nodes ** 3, dtype=np.int64)
    new_node[free_node] = np.arange(int(free_node.sum()))
    dof_map = (3 * new_node[:, None] + np.arange(3)[None, :]).ravel()
    dof_map[np.repeat(~free_node, 3)] = -1
    K = sp.csr_matrix((ndof, ndof))
    # assemble in chunks of elements to bound memory
    chunk = 65536
    for s0 in range(0, edofs.shape[0], chunk):
        ed = edofs[s0:s0 + chunk]
        r = np.repeat(ed, 24, axis=1).ravel()
        c = np.tile(ed, (1, 24)).ravel()
        v = np.tile(Ke.ravel(), ed.shape[0])
        K = K + sp.coo_matrix((v, (r, c)), shape=(ndof, ndof)).tocsr()
    keep = np.flatnonzero(dof_map >= 0)
    K = K[keep][:, keep]
    K = sp.csr_matrix(0.5 * (K + K.T))  # exact symmetry after floating-point assembly
    K.sort_indices()
    return _q1_pattern_with_values(nodes, K)


def _q1_pattern_with_values(nodes: int, K: sp.csr_matrix):
    """The clamped Q1 pattern (free nodes x = 1..nodes-1, y, z = 0..nodes-1; a node couples
    to the 27 nodes around it) in CSR with ascending columns, values looked up in K (which
    holds only the nonzero sums); every entry of K must lie in the pattern."""
    X, Y, Z = nodes - 1, nodes, nodes
    nn = X * Y * Z
    z, y, x = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    z, y, x = z.ravel(), y.ravel(), x.ravel()
    offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    valid = np.empty((nn, 27), bool)
    cnode = np.empty((nn, 27), np.int64)
    for o, (dz, dy, dx) in enumerate(offs):  # lexicographic (dz, dy, dx): ascending columns
        valid[:, o] = ((0 <= z + dz) & (z + dz < Z) & (0 <= y + dy) & (y + dy < Y)
                       & (0 <= x + dx) & (x + dx < X))
        cnode[:, o] = np.arange(nn) + (dz * Y + dy) * X + dx
    cols = 3 * cnode[:, :, None] + np.arange(3)[None, None, :]              # (nn, 27, 3)
    ci = np.broadcast_to(cols[:, None], (nn, 3, 27, 3))[
        np.broadcast_to(valid[:, None, :, None], (nn, 3, 27, 3))].astype(np.int64)
    lens = np.repeat(3 * valid.sum(axis=1), 3)
    n = 3 * nn
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    rows = np.repeat(np.arange(n, dtype=np.int64), lens)
    key = rows * n + ci
    del rows
    kr = np.repeat(np.arange(n, dtype=np.int64), np.diff(K.indptr))
    kkey = kr * n + K.indices.astype(np.int64)
    del kr
    pos = np.searchsorted(key, kkey)
    if not (pos < len(key)).all() or not np.array_equal(key[np.minimum(pos, len(key) - 1)], kkey):
        raise AssertionError("assembled entry outside the Q1 node-neighbour pattern")
    val = np.zeros(len(key), np.float64)
    val[pos] = K.data
    return rp.astype(np.int32), ci.astype(np.int32), val


def _exact_csr(n: int, r: np.ndarray, c: np.ndarray, v: np.ndarray):
    """CSR from duplicate-free triplets, keeping stored zeros (scipy would drop them)."""
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rp[1:])
    return rp.astype(np.int32), c.astype(np.int32), v.astype(np.float64)


def random_spd(n: int, avg_degree: float = 4.0, seed: int = 0, ties: bool = False,
               explicit_zeros: float = 0.0):
    """Random symmetric, strictly diagonally dominant (hence s.p.d.) sparse matrix.

    ties=True draws off-diagonal values from {-1, -2} so that many edge weights tie;
    explicit_zeros is the fraction of off-diagonal pairs stored with value 0.
    """
    rng = np.random.default_rng(seed)
    m = int(avg_degree * n / 2)
    a = rng.integers(0, n, size=m)
    b = rng.integers(0, n, size=m)
    keep = a != b
    a, b = np.minimum(a[keep], b[keep]), np.maximum(a[keep], b[keep])
    pairs = np.unique(a.astype(np.int64) * n + b)
    a, b = pairs // n, pairs % n
    if ties:
        w = -rng.integers(1, 3, size=len(a)).astype(np.float64)
    else:
        w = -rng.uniform(0.1, 1.0, size=len(a)) * rng.choice([1.0, -1.0], size=len(a), p=[0.8, 0.2])
    if explicit_zeros > 0:
        w[rng.random(len(a)) < explicit_zeros] = 0.0
    rowsum = np.bincount(a, weights=np.abs(w), minlength=n) + np.bincount(b, weights=np.abs(w), minlength=n)
    diag = rowsum + (1.0 if ties else rng.uniform(0.1, 1.0, size=n))
    d = np.arange(n, dtype=np.int64)
    return _exact_csr(n, np.concatenate([a, b, d]), np.concatenate([b, a, d]),
                      np.concatenate([w, w, diag]))


def random_spd_hubs(n: int, avg_degree: float = 4.0, n_hubs: int = 8, hub_degree: int = 300, seed: int = 0):
    """random_spd plus n_hubs vertices joined to hub_degree random others each: a few rows
    far longer than the mean, like the hub rows of a lognormal coarse level."""
    rng = np.random.default_rng(seed)
    m = int(avg_degree * n / 2)
    a = rng.integers(0, n, size=m)
    b = rng.integers(0, n, size=m)
    hubs = rng.choice(n, size=n_hubs, replace=False)
    a = np.concatenate([a, np.repeat(hubs, hub_degree)])
    b = np.concatenate([b, rng.integers(0, n, size=n_hubs * hub_degree)])
    keep = a != b
    a, b = np.minimum(a[keep], b[keep]), np.maximum(a[keep], b[keep])
    pairs = np.unique(a.astype(np.int64) * n + b)
    a, b = pairs // n, pairs % n
    w = -rng.uniform(0.1, 1.0, size=len(a))
    rowsum = np.bincount(a, weights=np.abs(w), minlength=n) + np.bincount(b, weights=np.abs(w), minlength=n)
    diag = rowsum + rng.uniform(0.1, 1.0, size=n)
    d = np.arange(n, dtype=np.int64)
    return _exact_csr(n, np.concatenate([a, b, d]), np.concatenate([b, a, d]),
                      np.concatenate([w, w, diag]))


def random_block3_spd(nbr: int, avg_blocks: float = 6.0, n_hubs: int = 3, hub_blocks: int = 80, seed: int = 0,
                      zero_frac: float = 0.1):
    """Random s.p.d. matrix of 3 nbr rows whose pattern is made of whole 3x3 blocks (block rows
    3b..3b+2 share their columns, in aligned triples), like a nodal 3D vector problem with
    interleaved unknowns: off-diagonal blocks U[-1, 1] with a fraction zero_frac of their
    entries exactly zero (stored), a few hub block rows far longer than the mean, and
    diagonal blocks made strictly diagonally dominant.  Bit-symmetric."""
    rng = np.random.default_rng(seed)
    m = int(avg_blocks * nbr / 2)
    a = rng.integers(0, nbr, size=m)
    b = rng.integers(0, nbr, size=m)
    hubs = rng.choice(nbr, size=n_hubs, replace=False)
    a = np.concatenate([a, np.repeat(hubs, hub_blocks)])
    b = np.concatenate([b, rng.integers(0, nbr, size=n_hubs * hub_blocks)])
    keep = a != b
    a, b = np.minimum(a[keep], b[keep]), np.maximum(a[keep], b[keep])
    pairs = np.unique(a.astype(np.int64) * nbr + b)
    a, b = pairs // nbr, pairs % nbr
    blk = rng.uniform(-1.0, 1.0, size=(len(a), 3, 3))
    blk[rng.random(blk.shape) < zero_frac] = 0.0
    rows, cols, vals = [], [], []
    ii, jj = np.meshgrid(np.arange(3), np.arange(3), indexing="ij")
    for (x, y, B) in ((a, b, blk), (b, a, blk.transpose(0, 2, 1))):
        rows.append((3 * x[:, None, None] + ii[None]).ravel())
        cols.append((3 * y[:, None, None] + jj[None]).ravel())
        vals.append(B.ravel())
    n = 3 * nbr
    r, c, v = np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)
    rowsum = np.bincount(r, weights=np.abs(v), minlength=n)
    D = rng.uniform(-0.2, 0.2, size=(nbr, 3, 3))
    D = 0.5 * (D + D.transpose(0, 2, 1))
    D[:, ii == jj] = 0.0
    dsum = np.abs(D).sum(axis=2).ravel()
    D[:, np.arange(3), np.arange(3)] = (rowsum + dsum + rng.uniform(0.1, 1.0, size=n)).reshape(nbr, 3)
    d = np.arange(nbr)
    r = np.concatenate([r, (3 * d[:, None, None] + ii[None]).ravel()])
    c = np.concatenate([c, (3 * d[:, None, None] + jj[None]).ravel()])
    v = np.concatenate([v, D.ravel()])
    return _exact_csr(n, r, c, v)


def smooth_vector_ones(n: int) -> np.ndarray:
    return np.ones(n, np.float64)


def smooth_vector_components(n: int, ncomp: int = 3, seed: int = 0) -> np.ndarray:
    """v_i = c_{i mod ncomp}, c ~ U[0.5, 1.5]^ncomp: rigid translations with seeded weights."""
    c = np.random.default_rng(seed).uniform(0.5, 1.5, size=ncomp)
    return c[np.arange(n) % ncomp].astype(np.float64)


def manufactured_rhs(rp, ci, val, seed: int = 0):
    """x* ~ U[-1, 1] (seeded) and b = A x* (row sums in CSR order)."""
    n = len(rp) - 1
    xs = np.random.default_rng(seed).uniform(-1.0, 1.0, size=n)
    a = sp.csr_matrix((val, ci, rp), shape=(n, n))
    return xs, a @ xs


def to_scipy(rp, ci, val) -> sp.csr_matrix:
    n = len(rp) - 1
    return sp.csr_matrix((val, ci, rp), shape=(n, n))


_FV_PATTERN_CACHE: dict = {}


def _fv_pattern(shape):
    """COO (rows, cols) of diffusion_fv's entries in its assembly order, the permutation that
    sorts them into CSR order, and the CSR (row_ptr, col)."""
    if shape in _FV_PATTERN_CACHE:
        return _FV_PATTERN_CACHE[shape]
    mz, my, mx = shape
    n = mz * my * mx
    idx = np.arange(n, dtype=np.int64).reshape(mz, my, mx)
    rows, cols = [], []
    for axis in (2, 1, 0):
        i0 = np.moveaxis(idx, axis, 0)
        a, b = i0[:-1].ravel(), i0[1:].ravel()
        rows += [a, b]
        cols += [b, a]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    perm = np.lexsort((c, r))
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=rp[1:])
    out = (perm, rp.astype(np.int32), c[perm].astype(np.int32))
    _FV_PATTERN_CACHE[shape] = out
    return out


def diffusion_fv_torch(kappa):
    """diffusion_fv as differentiable torch operations: returns (row_ptr, col, val) with
    row_ptr/col as numpy int32 and val a torch tensor on kappa's device and dtype, equal
    value for value to diffusion_fv(kappa) (the same operations in the same order)."""
    import torch
    mz, my, mx = kappa.shape
    perm, rp, ci = _fv_pattern((mz, my, mx))
    diag = torch.zeros_like(kappa)
    vals = []
    for axis in (2, 1, 0):
        k0 = kappa.movedim(axis, 0)
        d0 = diag.movedim(axis, 0)
        t = 2.0 * k0[:-1] * k0[1:] / (k0[:-1] + k0[1:])
        zero = torch.zeros_like(k0[:1])
        d0 = d0 + torch.cat([t, zero], 0)
        d0 = d0 + torch.cat([zero, t], 0)
        first = torch.zeros_like(k0)
        first[0] = 1.0
        last = torch.zeros_like(k0)
        last[-1] = 1.0
        d0 = d0 + first * (2.0 * k0)
        d0 = d0 + last * (2.0 * k0)
        diag = d0.movedim(0, axis)
        tv = (-t).reshape(-1)
        vals += [tv, tv]
    vals.append(diag.reshape(-1))
    coo = torch.cat(vals)
    return rp, ci, coo[torch.as_tensor(perm, device=coo.device)]

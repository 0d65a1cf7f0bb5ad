"""Pins of the oracle's l1-Jacobi smoother (Sec. 3.2), V-cycle (Sec. 2.1, Algorithm 1)
and flexible CG (Sec. 3.2, Algorithm 3) against textbook identities, scipy's CG and
direct solves (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from paper_1810_04221_gb300 import problems as P


def _hier(kind="diff", sweeps=2, coarse_max=30, **kw):
    if kind == "diff":
        rp, ci, val = P.lognormal_diffusion(8, seed=2)
    elif kind == "p2":
        rp, ci, val = P.poisson2d(16)
    else:
        rp, ci, val = P.random_spd(400, 5.0, seed=4)
    n = len(rp) - 1
    return (rp, ci, val), oracle.Hierarchy(rp, ci, val, np.ones(n), sweeps=sweeps,
                                           coarse_max=coarse_max, **kw)


def _dense_levels(H):
    Ls = [H.level(k) for k in range(H.nl)]
    A = [P.to_scipy(L["rp"], L["ci"], L["val"]).toarray() for L in Ls]
    Pm = [sp.csr_matrix((L["p"], (np.arange(L["n"]), L["agg"])),
                        shape=(L["n"], Ls[k + 1]["n"])).toarray() for k, L in enumerate(Ls[:-1])]
    D = [L["dl1"] for L in Ls]
    return A, Pm, D


def test_l1_jacobi_norms_and_contraction():
    (rp, ci, val), H = _hier("rand")
    A = P.to_scipy(rp, ci, val)
    L0 = H.level(0)
    assert np.allclose(L0["dl1"], np.asarray(abs(A).sum(axis=1)).ravel(), rtol=1e-15, atol=0)
    # l1-Jacobi is convergent for s.p.d. A: the A-norm of the error decreases every sweep
    n = len(rp) - 1
    xs = np.random.default_rng(0).standard_normal(n)
    b = A @ xs
    x = np.zeros(n)
    prev = np.sqrt((xs - x) @ (A @ (xs - x)))
    for _ in range(5):
        x = H.l1_jacobi(0, b, x, 1)
        cur = np.sqrt((xs - x) @ (A @ (xs - x)))
        assert cur < prev
        prev = cur
    # textbook identity: error propagation of s sweeps is (I - D^{-1} A)^s
    Ad = A.toarray()
    E = np.eye(n) - Ad / L0["dl1"][:, None]
    x0 = np.random.default_rng(1).standard_normal(n)
    x3 = H.l1_jacobi(0, b, x0, 3)
    assert np.abs((xs - x3) - np.linalg.matrix_power(E, 3) @ (xs - x0)).max() < 1e-12


@pytest.mark.parametrize("kind", ["diff", "p2", "rand"])
def test_coarsest_sweeps_map_is_symmetric(kind):
    """The coarsest level's 20 l1-Jacobi sweeps from zero are the linear map
    B = sum_{k<20} (I - D^-1 A)^k D^-1, and B is symmetric for symmetric A (it equals
    D^-1/2 p(D^-1/2 A D^-1/2) D^-1/2); a GPU may therefore build B on one triangle.  B is
    taken column by column from the oracle's own sweeps on unit vectors."""
    (rp, ci, val), H = _hier(kind)
    k = H.nl - 1
    A, _, D = _dense_levels(H)
    Ac, dc = A[k], D[k]
    nc = Ac.shape[0]
    assert 1 < nc <= 60
    Bm = np.empty((nc, nc))
    for c in range(nc):
        e = np.zeros(nc)
        e[c] = 1.0
        Bm[:, c] = H.l1_jacobi(k, e, np.zeros(nc), 20)
    scale = np.abs(Bm).max()
    assert np.abs(Bm - Bm.T).max() <= 1e-13 * scale
    M = np.eye(nc) - Ac / dc[:, None]
    closed, term = np.zeros((nc, nc)), np.diag(1.0 / dc)
    for _ in range(20):
        closed += term
        term = M @ term
    assert np.abs(Bm - closed).max() <= 1e-13 * scale
    # not a property every sweep count of every matrix shares: a nonsymmetric A breaks it
    An = Ac.copy()
    i, j = next((i, j) for i, j in zip(*np.nonzero(Ac)) if i != j)
    An[i, j] *= 1.5
    Mn = np.eye(nc) - An / dc[:, None]
    Bn, term = np.zeros((nc, nc)), np.diag(1.0 / dc)
    for _ in range(20):
        Bn += term
        term = Mn @ term
    assert np.abs(Bn - Bn.T).max() > 1e-6 * np.abs(Bn).max()


@pytest.mark.parametrize("kind,pre,post", [("diff", 1, 1), ("p2", 1, 1), ("rand", 2, 1)])
def test_vcycle_error_propagation_identity(kind, pre, post):
    """I - B A = (I - D^-1 A)^post (I - P B_c P^T A) (I - D^-1 A)^pre per level and
    I - B_c A_c = (I - D_c^-1 A_c)^coarse on the coarsest level (multigrid identity)."""
    _, H = _hier(kind, pre=pre, post=post, coarse_sweeps=20)
    A, Pm, D = _dense_levels(H)
    nl = H.nl
    assert nl >= 3
    B = [None] * nl
    nc = A[-1].shape[0]
    S = np.eye(nc) - A[-1] / D[-1][:, None]
    B[-1] = (np.eye(nc) - np.linalg.matrix_power(S, 20)) @ np.linalg.inv(A[-1])
    for k in range(nl - 2, -1, -1):
        n = A[k].shape[0]
        S = np.eye(n) - A[k] / D[k][:, None]
        C = np.eye(n) - Pm[k] @ B[k + 1] @ Pm[k].T @ A[k]
        E = np.linalg.matrix_power(S, post) @ C @ np.linalg.matrix_power(S, pre)
        B[k] = (np.eye(n) - E) @ np.linalg.inv(A[k])
    n = A[0].shape[0]
    R = np.random.default_rng(3).standard_normal((n, 4))
    for c in range(4):
        w = H.vcycle(R[:, c])
        ref = B[0] @ R[:, c]
        assert np.abs(w - ref).max() <= 1e-10 * np.abs(ref).max()


def test_vcycle_symmetric_positive():
    _, H = _hier("diff")
    n = H.level_n(0)
    rng = np.random.default_rng(5)
    for _ in range(3):
        x, y = rng.standard_normal(n), rng.standard_normal(n)
        bx, by = H.vcycle(x), H.vcycle(y)
        assert abs(bx @ y - x @ by) <= 1e-12 * abs(bx @ y) + 1e-14
        assert x @ bx > 0


@pytest.mark.parametrize("prec", [oracle.PREC_IDENTITY, oracle.PREC_L1JACOBI])
def test_fcg_matches_textbook_pcg(prec):
    """For a fixed s.p.d. preconditioner, FCG(1) reduces to the classic PCG (scipy.cg)."""
    (rp, ci, val), H = _hier("rand")
    A = P.to_scipy(rp, ci, val)
    n = A.shape[0]
    xs, b = P.manufactured_rhs(rp, ci, val, seed=1)
    x, st, it, rr, rt = H.pcg(b, rtol=1e-10, itmax=2000, prec=prec)
    assert st == oracle.OK
    count = [0]
    M = None
    if prec == oracle.PREC_L1JACOBI:
        d = H.level(0)["dl1"]
        M = spla.LinearOperator((n, n), matvec=lambda r: r / d)
    xref, info = spla.cg(A, b, rtol=1e-10, atol=0.0, maxiter=2000, M=M,
                         callback=lambda _: count.__setitem__(0, count[0] + 1))
    assert info == 0
    assert abs(it - count[0]) <= 1
    assert np.abs(x - xref).max() <= 1e-7 * np.abs(xref).max()


@pytest.mark.parametrize("kind", ["diff", "p2", "rand"])
def test_fcg_amg_solution_vs_direct(kind):
    (rp, ci, val), H = _hier(kind)
    A = P.to_scipy(rp, ci, val)
    xs, b = P.manufactured_rhs(rp, ci, val, seed=2)
    x, st, it, rr, rt = H.pcg(b, rtol=1e-10, itmax=500)
    assert st == oracle.OK and rr <= 1e-10
    assert rt <= 1e-9
    xd = spla.spsolve(A.tocsc(), b)
    assert np.abs(x - xd).max() <= 1e-7 * np.abs(xd).max()


def test_fcg_zero_rhs_and_itmax():
    _, H = _hier("p2")
    n = H.level_n(0)
    x, st, it, rr, rt = H.pcg(np.zeros(n))
    assert st == oracle.OK and it == 0 and np.all(x == 0)
    b = np.random.default_rng(0).standard_normal(n)
    x, st, it, rr, rt = H.pcg(b, rtol=1e-30, itmax=3)
    assert st == oracle.ERR_NOT_CONVERGED and it == 3


def test_fcg_poisson64_reference_iterations():
    """64^2 Poisson, 2 sweeps, coarse <= 40, rtol 1e-8: converges; the recursive and the
    true residual agree."""
    rp, ci, val = P.poisson2d(64)
    H = oracle.Hierarchy(rp, ci, val, np.ones(4096), sweeps=2, coarse_max=40)
    xs, b = P.manufactured_rhs(rp, ci, val, seed=0)
    x, st, it, rr, rt = H.pcg(b, rtol=1e-8)
    assert st == oracle.OK and 5 < it < 60
    assert abs(rr - rt) < 1e-10
    assert np.abs(x - xs).max() < 1e-5


@pytest.mark.parametrize("kind", ["diff", "p2"])
def test_wcycle_error_propagation_identity(kind):
    """W-cycle (two coarse cycles per level, Sec. 5.1): E_k = S^post (I - P (I - E_{k+1}^2)
    A_{k+1}^{-1} P^T A_k) S^pre, with E the error propagator I - B A of each level and
    E_coarsest = (I - D^-1 A)^sweeps."""
    _, H = _hier(kind, gamma=2)
    A, Pm, D = _dense_levels(H)
    nl = H.nl
    assert nl >= 3
    E = [None] * nl
    nc = A[-1].shape[0]
    E[-1] = np.linalg.matrix_power(np.eye(nc) - A[-1] / D[-1][:, None], 20)
    for k in range(nl - 2, -1, -1):
        n = A[k].shape[0]
        S = np.eye(n) - A[k] / D[k][:, None]
        Ec2 = E[k + 1] @ E[k + 1]
        Bc = (np.eye(A[k + 1].shape[0]) - Ec2) @ np.linalg.inv(A[k + 1])
        C = np.eye(n) - Pm[k] @ Bc @ Pm[k].T @ A[k]
        E[k] = S @ C @ S
    B0 = (np.eye(A[0].shape[0]) - E[0]) @ np.linalg.inv(A[0])
    r = np.random.default_rng(8).standard_normal(A[0].shape[0])
    w = H.vcycle(r)
    ref = B0 @ r
    assert np.abs(w - ref).max() <= 1e-10 * np.abs(ref).max()
    # the W-cycle is symmetric too
    y = np.random.default_rng(9).standard_normal(A[0].shape[0])
    assert abs(H.vcycle(r) @ y - r @ H.vcycle(y)) <= 1e-12 * abs(r @ H.vcycle(y)) + 1e-14


def test_wcycle_fewer_iterations_than_vcycle():
    """Sec. 5.1: the W-cycle needs fewer FCG iterations than the V-cycle.  (Its cost grows
    as 2^levels, so the hierarchy here is kept short.)"""
    rp, ci, val = P.poisson3d(16)
    n = len(rp) - 1
    xs, b = P.manufactured_rhs(rp, ci, val, seed=1)
    itv = oracle.Hierarchy(rp, ci, val, np.ones(n), sweeps=3, coarse_max=10).pcg(b, rtol=1e-8)[2]
    itw = oracle.Hierarchy(rp, ci, val, np.ones(n), sweeps=3, coarse_max=10, gamma=2).pcg(b, rtol=1e-8)[2]
    assert itw < itv


def test_dense_solve_gradient_vs_finite_differences():
    """dL/db = lambda and dL/dA_ij = -lambda_i x_j (oracle/gradient.py) against central
    differences of the dense solve, each entry of A perturbed on its own."""
    from oracle.gradient import solve_grad
    rng = np.random.default_rng(3)
    rp, ci, val = P.random_spd(30, 4.0, seed=8)
    A = P.to_scipy(rp, ci, val).toarray()
    b = rng.standard_normal(30)
    xt = rng.standard_normal(30)
    x, L, gb, gA = solve_grad(A, b, xt)
    h = 1e-6
    for i in rng.choice(30, 5, replace=False):
        e = np.zeros(30)
        e[i] = h
        fd = (solve_grad(A, b + e, xt)[1] - solve_grad(A, b - e, xt)[1]) / (2 * h)
        assert abs(fd - gb[i]) <= 1e-6 * max(1.0, abs(gb[i]))
    for k in rng.choice(len(ci), 8, replace=False):
        i = int(np.searchsorted(rp, k, side="right") - 1)
        j = int(ci[k])
        E = np.zeros_like(A)
        E[i, j] = h
        fd = (solve_grad(A + E, b, xt)[1] - solve_grad(A - E, b, xt)[1]) / (2 * h)
        assert abs(fd - gA[i, j]) <= 1e-6 * max(1.0, abs(gA[i, j]))


def test_diffusion_fv_torch_matches_numpy():
    import torch
    k = P.lognormal_kappa(6, seed=2)
    rp, ci, val = P.diffusion_fv(k)
    rp2, ci2, v2 = P.diffusion_fv_torch(torch.from_numpy(k))
    assert np.array_equal(rp, rp2) and np.array_equal(ci, ci2)
    assert np.array_equal(val.view(np.int64), v2.numpy().view(np.int64))

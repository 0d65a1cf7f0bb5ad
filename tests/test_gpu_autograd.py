"""GPU: the differentiable solve (x = A^{-1} b through AMG-preconditioned FCG, backward by
the adjoint solve on the same hierarchy and the sampled outer product on A's pattern).

References: the dense FP64 gradient of oracle/gradient.py on small problems, autograd of a
dense torch solve through the FV assembly (dL/dkappa on a 12^3 copy), and central finite
differences on 32 random kappa entries of the 96^3 lognormal problem.
"""
import numpy as np
import pytest
import torch

from oracle.gradient import solve_grad
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


def test_pattern_outer_bit_exact(B):
    rp, ci, val = P.random_spd(3001, 9.0, seed=4)
    rng = np.random.default_rng(1)
    lam, x = rng.standard_normal(3001), rng.standard_normal(3001)
    got = host(B.cwm_pattern_outer(*csr_dev(rp, ci, val)[:2], dev(lam), dev(x), alpha=-1.0))
    rows = np.repeat(np.arange(3001), np.diff(rp))
    ref = -1.0 * (lam[rows] * x[ci])
    assert np.array_equal(got.view(np.int64), ref.view(np.int64))


def test_autograd_matches_dense_gradient(B):
    from paper_1810_04221_gb300.autograd import amg_solve
    kappa = P.lognormal_kappa(12, seed=5)
    rp, ci, val = P.diffusion_fv(kappa)
    n = len(rp) - 1
    rng = np.random.default_rng(2)
    b, xt = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    x_ref, L_ref, gb_ref, gA_ref = solve_grad(P.to_scipy(rp, ci, val).toarray(), b, xt)
    d_rp, d_ci = dev(rp), dev(ci)
    v = dev(val).requires_grad_(True)
    bb = dev(b).requires_grad_(True)
    prm = B.amg_default_params(sweeps_per_level=3, coarse_max=50)
    x = amg_solve(d_rp, d_ci, v, bb, params=prm, rtol=1e-12)
    L = 0.5 * ((x - dev(xt)) ** 2).sum()
    L.backward()
    assert abs(L.item() - L_ref) <= 1e-9 * abs(L_ref)
    assert np.abs(host(bb.grad) - gb_ref).max() <= 1e-7 * np.abs(gb_ref).max()
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert np.abs(host(v.grad) - gA_ref[rows, ci]).max() <= 1e-7 * np.abs(gA_ref).max()


def test_autograd_kappa_dense_12(B):
    """dL/dkappa through the differentiable FV assembly vs a dense torch solve."""
    from paper_1810_04221_gb300.autograd import amg_solve
    k_np = P.lognormal_kappa(12, seed=6)
    n = k_np.size
    rng = np.random.default_rng(3)
    b, xt = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    # dense reference on the CPU
    kc = torch.from_numpy(k_np).requires_grad_(True)
    rp, ci, vc = P.diffusion_fv_torch(kc)
    Ad = torch.zeros(n, n, dtype=torch.float64)
    rows = torch.from_numpy(np.repeat(np.arange(n), np.diff(rp)))
    Ad = Ad.index_put((rows, torch.from_numpy(ci).long()), vc)
    xr = torch.linalg.solve(Ad, torch.from_numpy(b))
    Lr = 0.5 * ((xr - torch.from_numpy(xt)) ** 2).sum()
    Lr.backward()
    # AMG on the GPU
    kg = dev(k_np).requires_grad_(True)
    rp2, ci2, vg = P.diffusion_fv_torch(kg)
    x = amg_solve(dev(rp2), dev(ci2), vg, dev(b), params=B.amg_default_params(sweeps_per_level=3, coarse_max=50),
                  rtol=1e-12)
    L = 0.5 * ((x - dev(xt)) ** 2).sum()
    L.backward()
    g_ref = kc.grad.numpy()
    assert np.abs(host(kg.grad) - g_ref).max() <= 1e-6 * np.abs(g_ref).max()


def test_autograd_kappa_finite_differences_96(B):
    """96^3 lognormal (n = 884,736): autograd dL/dkappa vs central differences (relative
    step 1e-6) on 32 random cells.  The differences carry the noise of two independent
    solves to 1e-12 (about 1e-6 of the largest gradient entry), hence the absolute term;
    the dense 12^3 comparison above is the tight check."""
    from paper_1810_04221_gb300.autograd import amg_solve
    k_np = P.lognormal_kappa(96, seed=0)
    n = k_np.size
    rng = np.random.default_rng(0)
    b = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
    xt = torch.from_numpy(rng.uniform(-1, 1, n)).cuda()
    prm = B.amg_default_params(sweeps_per_level=3, coarse_max=1000, stall_ratio=1.2)
    rp, ci, _ = P.diffusion_fv_torch(torch.from_numpy(k_np[:1, :1, :1]))  # warm the pattern cache path
    kg = dev(k_np).requires_grad_(True)
    rp, ci, vg = P.diffusion_fv_torch(kg)
    d_rp, d_ci = dev(rp), dev(ci)

    def loss(k):
        _, _, vv = P.diffusion_fv_torch(k)
        x = amg_solve(d_rp, d_ci, vv, b, params=prm, rtol=1e-12)
        return 0.5 * ((x - xt) ** 2).sum()

    L = loss(kg)
    L.backward()
    g = kg.grad.reshape(-1)
    cells = rng.choice(n, 32, replace=False)
    rows = []
    with torch.no_grad():
        base = dev(k_np).reshape(-1)
        for c in cells:
            h = 1e-6 * float(base[c])
            kp = base.clone()
            kp[c] += h
            km = base.clone()
            km[c] -= h
            fd = (loss(kp.reshape(k_np.shape)).item() - loss(km.reshape(k_np.shape)).item()) / (2 * h)
            rows.append((int(c), fd, g[c].item()))
    gmax = g.abs().max().item()
    print("\n".join(f"cell {c}: fd {fd:.8e} autograd {ga:.8e}" for c, fd, ga in rows))
    for c, fd, ga in rows:
        assert abs(fd - ga) <= 1e-4 * abs(ga) + 1e-6 * gmax, (c, fd, ga, gmax)

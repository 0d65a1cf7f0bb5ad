"""amg_setup and amg_pcg_solve on host arrays (page-locked and pageable): the same hierarchy,
iterations and solution bits as the device-array path; cwm_copy in and out of the device at
every word width and alignment."""
import numpy as np
import pytest
import torch

from paper_1810_04221_gb300 import problems as P
from tests.gpu_util import bits_equal, host

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


def _inputs():
    rp, ci, val = P.elasticity_q1(8)
    n = len(rp) - 1
    v = P.smooth_vector_components(n, seed=1)
    rng = np.random.default_rng(5)
    return [rp.astype(np.int32), ci.astype(np.int32), val, v, rng.uniform(-1, 1, n), rng.uniform(-0.1, 0.1, n)]


def _run(arrays, where, fp32):
    """Setup + solve with every array placed on `where`: cuda, pinned or pageable."""
    ts = [torch.from_numpy(np.ascontiguousarray(a)) for a in arrays]
    if where == "cuda":
        ts = [t.cuda() for t in ts]
    elif where == "pinned":
        ts = [t.pin_memory() for t in ts]
    rp, ci, val, v, b, x = ts
    prm = B.amg_default_params(sweeps_per_level=2, coarse_max=40, vcycle_fp32=fp32)
    h = B.amg_setup(rp, ci, val, v, prm)
    levels = [B.amg_level_info(h, k) for k in range(B.amg_num_levels(h))]
    st, info = B.amg_pcg_solve(h, b, x, rtol=1e-8, itmax=500)
    torch.cuda.synchronize()
    h.free()
    return host(x) if where == "cuda" else x.numpy().copy(), info, levels, st


@pytest.mark.parametrize("fp32", [0, 1])
@pytest.mark.parametrize("where", ["pinned", "pageable"])
def test_host_arrays_match_device_arrays(where, fp32):
    arrays = _inputs()
    x_d, info_d, lev_d, st_d = _run(arrays, "cuda", fp32)
    x_h, info_h, lev_h, st_h = _run(arrays, where, fp32)
    assert st_d == st_h == B.AMG_OK
    assert lev_h == lev_d
    assert info_h["iters"] == info_d["iters"]
    assert bits_equal(x_h, x_d)


def test_host_solution_written_back_on_repeated_solves():
    """Solves in a row on one handle with host b and x: the handle's device copies are
    refreshed from the caller's arrays on every call, and x is written back every time
    (itmax = 0 returns the initial guess unchanged)."""
    arrays = _inputs()
    rp, ci, val, v, b, x0 = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in arrays]
    h = B.amg_setup(rp, ci, val, v, B.amg_default_params(sweeps_per_level=2, coarse_max=40))
    x = x0.clone().pin_memory()
    st, info1 = B.amg_pcg_solve(h, b, x, rtol=1e-10, itmax=500)
    assert st == B.AMG_OK and info1["iters"] > 0
    x1 = x.numpy().copy()
    x.copy_(x0)
    st, info2 = B.amg_pcg_solve(h, b, x, rtol=1e-10, itmax=0)
    assert st == B.AMG_ERR_NOT_CONVERGED and info2["iters"] == 0
    assert bits_equal(x.numpy(), x0.numpy())
    b2 = (2.0 * b).pin_memory()
    x.zero_()
    st, info3 = B.amg_pcg_solve(h, b2, x, rtol=1e-10, itmax=500)
    assert st == B.AMG_OK and info3["iters"] > 0
    assert np.allclose(x.numpy(), 2.0 * x1, rtol=0, atol=1e-6 * np.abs(x1).max())
    h.free()


@pytest.mark.parametrize("where", ["pinned", "pageable"])
@pytest.mark.parametrize("offset,size", [(0, 1 << 20), (8, 4000), (4, 1002), (3, 1001), (0, 0)])
def test_cwm_copy_round_trip(where, offset, size):
    rng = np.random.default_rng(size + offset)
    src_h = torch.from_numpy(rng.integers(0, 256, size + 64, dtype=np.uint8))
    dst_h = torch.zeros(size + 64, dtype=torch.uint8)
    if where == "pinned":
        src_h, dst_h = src_h.pin_memory(), dst_h.pin_memory()
    d = torch.full((size + 32,), 7, dtype=torch.uint8, device="cuda")
    B.cwm_copy(d[16:16 + size], src_h[offset:offset + size])
    B.cwm_copy(dst_h[offset + 1:offset + 1 + size], d[16:16 + size])
    torch.cuda.synchronize()
    assert np.array_equal(host(d[16:16 + size]), src_h[offset:offset + size].numpy())
    assert np.all(host(d[:16]) == 7) and np.all(host(d[16 + size:]) == 7)
    out = dst_h.numpy()
    assert np.array_equal(out[offset + 1:offset + 1 + size], src_h[offset:offset + size].numpy())
    assert not out[:offset + 1].any() and not out[offset + 1 + size:].any()

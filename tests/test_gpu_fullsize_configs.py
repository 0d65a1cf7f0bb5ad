"""GPU: the other benchmark configurations at full size, against the oracle run at the
same size -- 3D lognormal FV diffusion 160^3 (log-kappa N(0, 2^2), 3 sweeps per level,
coarse n <= 1000, stall ratio 1.2) and Q1 elasticity on 64^3 nodes (2 sweeps per level,
coarse n <= 1000; the assembled pattern with its stored zeros, 60,756,300 entries), in the
launch configuration bench.py times (FP64 setup, FP32 V-cycle in
FP64 FCG).

Every level of the hierarchy is compared bit for bit (SHA-256 digests of the CSR arrays,
smooth vectors, aggregates and prolongator values); the FCG with the FP32 V-cycle must
reach 1e-8 within one iteration of the oracle's FP64 run and agree with its solution to
1e-6 relative.  The two oracle runs (one to three minutes each) go to spawned worker processes
when the module starts.
"""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest
import torch

import bench
from tests import fullsize_oracle as FO
from tests.gpu_util import csr_dev, dev, host

pytestmark = pytest.mark.gpu
WORKLOADS = ["lognormal_160", "elasticity_64"]


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_04221_gb300 import binding, build
    build.build()
    binding.load()
    return binding


@pytest.fixture(scope="module")
def oracle_runs():
    ex = cf.ProcessPoolExecutor(max_workers=len(WORKLOADS), mp_context=mp.get_context("spawn"))
    futs = {w: ex.submit(FO.run, w) for w in WORKLOADS}
    yield futs
    ex.shutdown(wait=True)


@pytest.mark.parametrize("workload", WORKLOADS)
def test_fullsize_config_vs_oracle(B, oracle_runs, workload):
    desc, mat, v, b, xs, sweeps, cmax, fp32, extra = bench.workload(workload)
    n = len(mat[0]) - 1
    prm = B.amg_default_params(sweeps_per_level=sweeps, coarse_max=cmax, vcycle_fp32=int(fp32), check_input=0,
                               **extra)
    h = B.amg_setup(*csr_dev(*mat), dev(v), prm)
    try:
        got = []
        for k in range(B.amg_num_levels(h)):
            L = B.amg_level_export(h, k)
            lev = {key: (None if L[key] is None else host(L[key])) for key in ("rp", "ci", "val", "v", "agg", "p")}
            got.append(FO.level_digests(lev))
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, info = B.amg_pcg_solve(h, dev(b), x, rtol=1e-8)
    finally:
        h.free()
    ref = oracle_runs[workload].result()
    assert len(got) == len(ref["levels"])
    for k, (g, r) in enumerate(zip(got, ref["levels"])):
        assert g == tuple(r), f"level {k} differs"
    assert st == B.AMG_OK and ref["status"] == 0
    assert abs(info["iters"] - ref["iters"]) <= 1
    assert info["rel_res_true"] <= 2e-8
    xr = ref["x"]
    assert np.abs(host(x) - xr).max() <= 1e-6 * np.abs(xr).max()

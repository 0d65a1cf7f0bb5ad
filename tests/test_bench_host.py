"""bench.py's host logic on CPU: the workloads' sizes against their closed forms and
right-hand sides, the roofline peak lookup, and the ncu traffic lookup, which must go
stale (None) once the kernel source differs from the one the counters were taken on."""
import hashlib
import json

import numpy as np
import scipy.sparse as sp

import bench


def _csr(mat):
    rp, ci, val = mat
    n = len(rp) - 1
    return sp.csr_matrix((val, ci, rp), shape=(n, n))


def test_poisson_workloads_closed_forms():
    # m^d grid points, 2d+1 entries per row less one per missing neighbour on each face
    _, mat, v, b, xs, sweeps, cmax, fp32, extra = bench.workload("poisson2d_64")
    n = 64 ** 2
    assert len(mat[0]) - 1 == n and len(mat[1]) == 5 * n - 4 * 64 == 20224
    assert (sweeps, cmax, fp32, extra) == (2, 40, False, {})
    assert np.allclose(_csr(mat) @ xs, b, rtol=0, atol=1e-12)
    assert np.array_equal(v, np.ones(n))
    _, mat, v, b, xs, sweeps, cmax, fp32, extra = bench.workload("poisson3d_128")
    n = 128 ** 3
    assert len(mat[0]) - 1 == n and len(mat[1]) == 7 * n - 6 * 128 ** 2 == 14581760
    assert (sweeps, cmax, fp32, extra) == (3, 1000, False, {})
    assert np.abs(xs).max() <= 1.0
    assert np.allclose(_csr(mat) @ xs, b, rtol=0, atol=1e-11)


def test_lognormal_workload_shape():
    _, mat, v, b, xs, sweeps, cmax, fp32, extra = bench.workload("lognormal_160")
    n = 160 ** 3
    assert len(mat[0]) - 1 == n and len(mat[1]) == 7 * n - 6 * 160 ** 2 == 28518400
    assert (sweeps, cmax, fp32, extra) == (3, 1000, True, {"stall_ratio": 1.2})
    A = _csr(mat)
    assert (A.diagonal() > 0).all()
    assert abs(A - A.T).max() == 0.0  # bit-symmetric, as amg_setup requires


def test_peaks_measured_and_fallback(tmp_path, monkeypatch):
    f = tmp_path / "peaks.json"
    f.write_text(json.dumps({"hbm_gbs": 1234.5}))
    monkeypatch.setattr(bench, "PEAKS_FILE", str(f))
    assert bench._peaks() == (1234.5, "measured")
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "absent.json"))
    assert bench._peaks() == (bench.FALLBACK_HBM_GBS, "fallback")


def test_traffic_lookup_goes_stale_with_the_source(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    entry = {"kernel": "k", "source": str(src), "dram_bytes_per_launch": 1.5e8,
             "source_sha256": hashlib.sha256(src.read_bytes()).hexdigest()}
    tf = tmp_path / "traffic.json"
    tf.write_text(json.dumps({"poisson3d_128": {"spmv_dots": entry}}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tf))
    assert bench._traffic_for("spmv_dots", "poisson3d_128") == 1.5e8
    assert bench._traffic_for("jacobi@0", "poisson3d_128") is None  # no capture for this class
    assert bench._traffic_for("spmv_dots", "lognormal_160") is None  # captured on another workload
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench._traffic_for("spmv_dots", "poisson3d_128") is None  # the kernel changed since the capture


def test_committed_traffic_entries_are_well_formed():
    with open(bench.TRAFFIC_FILE) as f:
        d = json.load(f)
    assert "spmv_dots_b3" in d["elasticity_64"]
    for wl, classes in d.items():
        assert wl in bench.WORKLOADS
        for cls, e in classes.items():
            assert set(e) >= {"kernel", "source", "source_sha256", "dram_bytes_per_launch", "profile"}
            assert len(e["source_sha256"]) == 64 and e["dram_bytes_per_launch"] > 0
            with open(f"{bench.ROOT}/{e['profile']}") as p:
                assert e["kernel"] in p.read()


def test_elasticity_workload_shape():
    """The default workload: Q1 elasticity on 64^3 nodes with the x = 0 face eliminated,
    the assembled pattern's stored zeros included, body force b ~ U[-1, 1]."""
    _, mat, v, b, xs, sweeps, cmax, fp32, extra = bench.workload("elasticity_64")
    n = 3 * 63 * 64 ** 2
    assert len(mat[0]) - 1 == n == 774144 and len(mat[1]) == 60756300
    assert (sweeps, cmax, fp32, extra) == (2, 1000, True, {})
    assert xs is None and b.shape == (n,) and np.abs(b).max() <= 1.0
    assert np.array_equal(b, np.random.default_rng(0).uniform(-1.0, 1.0, size=n))
    c = v[:3]
    assert np.array_equal(v, np.tile(c, n // 3)) and (0.5 <= c).all() and (c <= 1.5).all()


def test_cpu_samples_are_coarser_instances():
    """Every workload's CPU sample is a workload of the same family with no more entries."""
    for name, sample in bench.CPU_SAMPLE.items():
        assert name.split("_")[0] == sample.split("_")[0]
        assert int(sample.split("_")[1]) <= int(name.split("_")[1])


def test_both_arms_share_the_config_keys():
    a = bench.bench_config("elasticity_64", 10, 20, "d", 2, 1000, 1e-8, True, 1)
    assert set(a) == {"workload", "desc", "n", "nnz", "sweeps_per_level", "coarse_max", "rtol", "vcycle_fp32",
                      "l2", "parallelism"}


def test_class_rooflines():
    tr = [{"name": "spmv_dots", "launches": 2, "total_ms": 0.2, "bytes": 1.0e9},
          {"name": "weights", "launches": 0, "total_ms": 0.0, "bytes": 0.0}]
    out = bench.class_rooflines(tr, 5000.0)
    assert len(out) == 1 and out[0]["avg_launch_us"] == 100.0
    assert out[0]["achieved_gbs"] == 5000.0 and out[0]["frac"] == 1.0


def test_fp64_fractions():
    cls = [{"kernel": "spmv_dots_b3", "avg_launch_us": 100.0}, {"kernel": "weights@0", "avg_launch_us": 50.0},
           {"kernel": "residual@0", "avg_launch_us": 10.0}]
    out = bench.fp64_fractions(cls, n=1000, nnz=10000, nnz_nonzero=9000, r_fma=1e9, r_div=1e8)
    assert [o["kernel"] for o in out] == ["spmv_dots_b3", "weights@0"]
    assert abs(out[0]["fp64_us"] - 13.0) < 1e-9 and abs(out[0]["fp64_frac"] - 0.13) < 1e-9
    # 4000 edges x 4 / 1e9 s = 16 us (the division runs on the integer pipes)
    assert abs(out[1]["fp64_us"] - 16.0) < 1e-9 and abs(out[1]["fp64_frac"] - 0.32) < 1e-9
    # rows averaging more than 32 slots: every slot evaluated, 8000 x 4 / 1e9 s = 32 us
    out = bench.fp64_fractions(cls, n=1000, nnz=40000, nnz_nonzero=9000, r_fma=1e9, r_div=1e8)
    assert abs(out[1]["fp64_us"] - 32.0) < 1e-9

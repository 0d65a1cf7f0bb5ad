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
    tf.write_text(json.dumps({"spmv_dots": entry}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tf))
    assert bench._traffic_for("spmv_dots") == 1.5e8
    assert bench._traffic_for("jacobi@0") is None  # no capture for this class
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench._traffic_for("spmv_dots") is None  # the kernel changed since the capture


def test_committed_traffic_entries_are_well_formed():
    with open(bench.TRAFFIC_FILE) as f:
        d = json.load(f)
    assert "spmv_dots" in d
    for cls, e in d.items():
        assert set(e) >= {"kernel", "source", "source_sha256", "dram_bytes_per_launch", "profile"}
        assert len(e["source_sha256"]) == 64 and e["dram_bytes_per_launch"] > 0
        with open(f"{bench.ROOT}/{e['profile']}") as p:
            assert e["kernel"] in p.read()

"""Oracle side of the full-size configuration tests, run in a spawned worker process.

Builds the oracle hierarchy and FCG solve of a bench workload and returns SHA-256 digests
of every level's arrays (so that no multi-gigabyte array crosses the process boundary),
the iteration count and the solution.  Test infrastructure only.
"""
from __future__ import annotations

import hashlib
import os
import sys

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def level_digests(level: dict) -> tuple:
    """(n, nnz, rp, ci, val, v, agg, p) with the arrays as digests (agg, p: None on the
    coarsest level)."""
    agg, p = level.get("agg"), level.get("p")
    return (len(level["rp"]) - 1, len(level["ci"]), digest(level["rp"]), digest(level["ci"]), digest(level["val"]),
            digest(level["v"]), None if agg is None else digest(agg), None if p is None else digest(p))


def run(workload: str) -> dict:
    import bench
    import oracle
    desc, mat, v, b, xs, sweeps, cmax, fp32, extra = bench.workload(workload)
    H = oracle.Hierarchy(*mat, v, sweeps=sweeps, coarse_max=cmax, stall_ratio=extra.get("stall_ratio", 0.0))
    levels = [level_digests(H.level(k)) for k in range(H.nl)]
    x, st, it, rr, rt = H.pcg(b, rtol=1e-8)
    H.close()
    return {"levels": levels, "status": st, "iters": it, "x": x, "rel_res_true": rt}

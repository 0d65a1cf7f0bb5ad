"""Writes ``oracle_digests.json``: SHA-256 digests of every level the oracle builds for a
few seeded inputs (level arrays of Sec. 2.1/2.2: A^k in CSR, v^k, and the aggregation P^k
as column and value per row), the hierarchy statistics of Sec. 5.2, and the FCG iteration
count and solution digest of Algorithm 3.

The file guards the oracle against silent change.  When the oracle's arithmetic changes on
purpose, rerun this script (``python tests/golden/make_golden.py``) and name, in the commit
message, the passage of the paper, or the reading of it, that justifies the change.  Only
``oracle/`` and the seeded input generators are called; no value comes from the CUDA path.
The inputs avoid transcendental functions (their results may differ between platforms'
math libraries); the oracle itself is IEEE arithmetic with FMA contraction off, and
``sqrt``, which IEEE rounds exactly.
"""
import hashlib
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_1810_04221_gb300 import problems as P  # noqa: E402

OUT = os.path.join(HERE, "oracle_digests.json")

# name -> (generator, sweeps per level, coarse_max)
CASES = {
    "poisson2d_64_s2": (lambda: P.poisson2d(64), 2, 40),
    "poisson3d_24_s3": (lambda: P.poisson3d(24), 3, 20),
    "random_spd_2000_s2": (lambda: P.random_spd(2000, 6.0, seed=3), 2, 40),
    "random_spd_ties_1500_s3": (lambda: P.random_spd(1500, 5.0, seed=4, ties=True), 3, 30),
}


def _sha(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def digest(name: str) -> dict:
    gen, sweeps, cmax = CASES[name]
    rp, ci, val = gen()
    n = len(rp) - 1
    H = oracle.Hierarchy(rp, ci, val, np.ones(n), sweeps=sweeps, coarse_max=cmax)
    try:
        levels = []
        for k in range(H.nl):
            L = H.level(k)
            e = {"n": int(H.level_n(k)), "nnz": int(H.level_nnz(k)),
                 "A": _sha(L["rp"], L["ci"], L["val"]), "v": _sha(L["v"])}
            if k < H.nl - 1:
                e["P"] = _sha(L["agg"], L["p"])
            levels.append(e)
        vc, cr = H.stats()
        _, b = P.manufactured_rhs(rp, ci, val, seed=0)
        x, st, it, _, _ = H.pcg(b, rtol=1e-8, itmax=500)
        return {"nl": int(H.nl), "vcmplx": float(vc).hex(), "cratio": float(cr).hex(), "levels": levels,
                "pcg_status": int(st), "pcg_iters": int(it), "pcg_x": _sha(x)}
    finally:
        H.close()


def main():
    out = {name: digest(name) for name in CASES}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(f"wrote {OUT}")


if __name__ == "__main__":
    main()

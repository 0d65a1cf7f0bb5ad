"""The oracle against its stored digests (tests/golden/oracle_digests.json, written by
tests/golden/make_golden.py from the oracle alone): every level's A^k, v^k and P^k, the
Sec. 5.2 statistics and the FCG result of Algorithm 3 for four seeded inputs.  A failure
means the oracle's arithmetic changed; the fixture is regenerated only on purpose, with the
passage that justifies the change named in the commit message.

Two cases also carry hand-derived values that pin the digests to the mathematics:
the 2D Poisson 64^2 hierarchy has the closed form 4096 -> 1024 -> 256 -> 64 -> 16 (2x2
aggregates on every level), and its statistics follow from the level sizes alone."""
import json
import os

import pytest

from tests.golden import make_golden as G

with open(G.OUT) as _f:
    GOLDEN = json.load(_f)


@pytest.mark.parametrize("name", sorted(G.CASES))
def test_oracle_matches_stored_digests(name):
    got = G.digest(name)
    want = GOLDEN[name]
    assert got["nl"] == want["nl"]
    for k, (g, w) in enumerate(zip(got["levels"], want["levels"])):
        assert g == w, f"level {k}"
    assert (got["vcmplx"], got["cratio"]) == (want["vcmplx"], want["cratio"])
    assert (got["pcg_status"], got["pcg_iters"], got["pcg_x"]) == (want["pcg_status"], want["pcg_iters"],
                                                                    want["pcg_x"])


def test_stored_poisson2d_closed_form():
    """The stored 64^2 hierarchy is the closed form: n = (64/2^k)^2, nnz = 5m^2 - 4m,
    Vcmplx = sum nnz / nnz_0 and cratio = (1/nl) * sum of the four ratios 4 (Sec. 5.2)."""
    g = GOLDEN["poisson2d_64_s2"]
    ms = [64, 32, 16, 8, 4]
    assert g["nl"] == 5
    assert [lv["n"] for lv in g["levels"]] == [m * m for m in ms]
    assert [lv["nnz"] for lv in g["levels"]] == [5 * m * m - 4 * m for m in ms]
    assert float.fromhex(g["vcmplx"]) == pytest.approx(sum(5 * m * m - 4 * m for m in ms) / 20224, abs=1e-15)
    assert float.fromhex(g["cratio"]) == 16.0 / 5.0


def test_generator_writes_only_oracle_values():
    """The fixture's writer imports the oracle and the input generators, nothing from the
    CUDA path."""
    src = open(os.path.join(os.path.dirname(G.OUT), "make_golden.py")).read()
    assert "binding" not in src and "csrc" not in src and "libcwmamg" not in src

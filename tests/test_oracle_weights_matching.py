"""Pins of the oracle's edge weights and matching against closed forms, brute force
and the greedy/locally-dominant characterisation (CPU only).

Edge weight (Sec. 2.2; the formula itself comes from the method's statement of C(A, v)):
    c_ab = 1 - 2 a_ab v_a v_b / (a_aa v_a^2 + a_bb v_b^2).
Matching (Sec. 3.1): Suitor, a 1/2-approximation of the maximum weight matching of Sec. 2.2.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1810_04221_gb300 import problems as P


def _edges(rp, ci, w):
    """Upper-triangle eligible edges as {(a, b): c}."""
    out = {}
    for i in range(len(rp) - 1):
        for k in range(rp[i], rp[i + 1]):
            j = int(ci[k])
            if j > i and w[k] > 0:
                out[(i, j)] = float(w[k])
    return out


# ---------------------------------------------------------------- weights ----

def test_weight_hand_example_2x2():
    # A = [[2, -1], [-1, 3]], v = (1, 2):  c = 1 + 2*1*2/(2*1 + 3*4) = 1 + 4/14 = 9/7.
    rp = np.array([0, 2, 4], np.int32)
    ci = np.array([0, 1, 0, 1], np.int32)
    val = np.array([2.0, -1.0, -1.0, 3.0])
    w = oracle.edge_weights(rp, ci, val, np.array([1.0, 2.0]))
    assert w[0] == 0.0 and w[3] == 0.0  # diagonal slots carry no edge
    assert w[1] == w[2]
    assert abs(w[1] - 9.0 / 7.0) < 1e-15
    # swapping v swaps the roles of a_aa and a_bb: 1 + 4/(2*4 + 3*1) = 15/11
    w2 = oracle.edge_weights(rp, ci, val, np.array([2.0, 1.0]))
    assert abs(w2[1] - 15.0 / 11.0) < 1e-15


def test_weight_positive_coupling_and_negative_v():
    # a_01 = +1 (positive coupling), v = (1, -1): c = 1 - 2*1*1*(-1)/(4+4) = 1.25
    rp = np.array([0, 2, 4], np.int32)
    ci = np.array([0, 1, 0, 1], np.int32)
    val = np.array([4.0, 1.0, 1.0, 4.0])
    w = oracle.edge_weights(rp, ci, val, np.array([1.0, -1.0]))
    assert w[1] == 1.25
    # same v sign: c = 1 - 2/8 = 0.75
    w = oracle.edge_weights(rp, ci, val, np.array([1.0, 1.0]))
    assert w[1] == 0.75


def test_weight_ineligible_cases():
    # explicit zero, v_i = v_j = 0 (den 0) and a non-positive weight are ineligible
    rp = np.array([0, 3, 6, 9], np.int32)
    ci = np.array([0, 1, 2, 0, 1, 2, 0, 1, 2], np.int32)
    val = np.array([2.0, 0.0, -1.0, 0.0, 2.0, -1.0, -1.0, -1.0, 2.0])
    w = oracle.edge_weights(rp, ci, val, np.array([0.0, 0.0, 1.0]))
    assert w[1] == 0 and w[3] == 0            # stored zero
    assert w[2] > 0 and w[6] == w[2]          # v_0 = 0 but den = a_22 > 0: c = 1
    assert w[2] == 1.0
    # a 2x2 block that is not p.d. (a_01 = +3, a_00 = a_11 = 1, v = 1): c = 1 - 6/2 = -2 -> ineligible
    rp2 = np.array([0, 2, 4], np.int32)
    ci2 = np.array([0, 1, 0, 1], np.int32)
    w2 = oracle.edge_weights(rp2, ci2, np.array([1.0, 3.0, 3.0, 1.0]), np.ones(2))
    assert w2[1] == 0.0 and w2[2] == 0.0


def test_weight_missing_or_nonpositive_diagonal_rejected():
    rp = np.array([0, 2, 4], np.int32)
    ci = np.array([0, 1, 0, 1], np.int32)
    with pytest.raises(ValueError):
        oracle.edge_weights(rp, ci, np.array([0.0, -1.0, -1.0, 2.0]), np.ones(2))


def test_weight_poisson_closed_forms():
    rp, ci, val = P.poisson2d(8)
    w = oracle.edge_weights(rp, ci, val, np.ones(64))
    assert set(np.unique(w)) == {0.0, 1.25}   # 1 + 2/(4+4)
    rp, ci, val = P.poisson3d(6)
    w = oracle.edge_weights(rp, ci, val, np.ones(216))
    assert set(np.unique(w)) == {0.0, 1.0 + 2.0 / 12.0}


def test_weight_range_and_bit_symmetry_random_spd():
    for seed in range(5):
        rp, ci, val = P.random_spd(300, 6.0, seed=seed)
        v = np.random.default_rng(seed).uniform(-2, 2, 300)
        w = oracle.edge_weights(rp, ci, val, v)
        off = ci != np.repeat(np.arange(300), np.diff(rp))
        # s.p.d. 2x2 principal blocks => 0 < c < 2 (AM-GM)
        assert np.all((w[off] > 0) & (w[off] < 2))
        e = _edges(rp, ci, w)
        for i in range(300):
            for k in range(rp[i], rp[i + 1]):
                j = int(ci[k])
                if j < i:
                    assert w[k] == e[(j, i)]


def test_weight_exact_rational():
    # the formula in exact rational arithmetic on a random small matrix with dyadic data
    rng = np.random.default_rng(7)
    rp, ci, val = P.random_spd(40, 5.0, seed=3, ties=True)
    v = rng.integers(-4, 5, 40).astype(float) / 4.0
    w = oracle.edge_weights(rp, ci, val, v)
    d = {i: Fraction(val[k]) for i in range(40) for k in range(rp[i], rp[i + 1]) if ci[k] == i}
    for i in range(40):
        for k in range(rp[i], rp[i + 1]):
            j = int(ci[k])
            if j == i:
                continue
            den = d[i] * Fraction(v[i]) ** 2 + d[j] * Fraction(v[j]) ** 2
            if den == 0:
                assert w[k] == 0
                continue
            c = 1 - 2 * Fraction(val[k]) * Fraction(v[i]) * Fraction(v[j]) / den
            if c <= 0:
                assert w[k] == 0
            else:
                assert abs(Fraction(w[k]) - c) <= Fraction(1, 2 ** 50) * abs(c)


# --------------------------------------------------------------- matching ----

def _check_greedy_characterisation(rp, ci, w, mate):
    """mate is the greedy matching under key (c, b, a) iff it is a matching and every
    unmatched edge has an adjacent matched edge with a larger key."""
    n = len(mate)
    for i in range(n):
        if mate[i] >= 0:
            assert mate[mate[i]] == i and mate[i] != i
    E = _edges(rp, ci, w)
    key = {e: (c, e[1], e[0]) for e, c in E.items()}
    for (a, b) in E:
        assert (mate[a] == b) == (mate[b] == a)
    for (a, b), k in key.items():
        if mate[a] == b:
            continue
        dom = []
        for x in (a, b):
            if mate[x] >= 0:
                y = mate[x]
                dom.append(key[(min(x, y), max(x, y))])
        assert dom and max(dom) > k, f"edge {(a, b)} not dominated"


def _max_weight_matching_brute(n, E):
    best = [0.0]
    elist = sorted(E.items())

    def rec(idx, used, total):
        if total + sum(c for _, c in elist[idx:]) <= best[0]:
            return
        if idx == len(elist):
            best[0] = max(best[0], total)
            return
        (a, b), c = elist[idx]
        if not (used >> a) & 1 and not (used >> b) & 1:
            rec(idx + 1, used | (1 << a) | (1 << b), total + c)
        rec(idx + 1, used, total)

    rec(0, 0, 0.0)
    return best[0]


@pytest.mark.parametrize("seed", range(12))
def test_matching_half_approx_vs_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(5, 12))
    rp, ci, val = P.random_spd(n, 3.0, seed=seed, ties=bool(seed % 3 == 0))
    v = rng.uniform(0.5, 1.5, n)
    w = oracle.edge_weights(rp, ci, val, v)
    E = _edges(rp, ci, w)
    mate = oracle.greedy_match(rp, ci, w)
    got = sum(c for (a, b), c in E.items() if mate[a] == b)
    opt = _max_weight_matching_brute(n, E)
    assert got >= 0.5 * opt - 1e-12
    _check_greedy_characterisation(rp, ci, w, mate)


@pytest.mark.parametrize("seed,ties", [(0, False), (1, True), (2, False), (3, True)])
def test_greedy_equals_sequential_suitor(seed, ties):
    rp, ci, val = P.random_spd(2000, 7.0, seed=seed, ties=ties)
    v = np.random.default_rng(seed).uniform(0.2, 2.0, 2000) if not ties else np.ones(2000)
    w = oracle.edge_weights(rp, ci, val, v)
    m1 = oracle.greedy_match(rp, ci, w)
    m2 = oracle.suitor_match(rp, ci, w)
    assert np.array_equal(m1, m2)
    _check_greedy_characterisation(rp, ci, w, m1)


def _python_greedy(edges, n, key):
    """Textbook greedy matching: scan the edges in decreasing key, take an edge whose ends
    are both free."""
    mate = [-1] * n
    for (a, b) in sorted(edges, key=lambda e: key(edges[e], e[0], e[1]), reverse=True):
        if mate[a] < 0 and mate[b] < 0:
            mate[a], mate[b] = b, a
    return np.array(mate)


@pytest.mark.parametrize("seed", range(6))
def test_greedy_equals_python_greedy_with_ties(seed):
    """The oracle's matching equals a plain Python greedy under the key (c, b, a).  Ties are
    frequent here (weights from two values); the key compared as (c, a, b) gives the same
    matching too: at a shared vertex both orders compare the other endpoint, and the greedy
    result depends only on how adjacent edges compare."""
    rp, ci, val = P.random_spd(300, 6.0, seed=40 + seed, ties=True)
    w = oracle.edge_weights(rp, ci, val, np.ones(300))
    edges = _edges(rp, ci, w)
    assert len(set(edges.values())) < len(edges) // 4  # many ties
    got = oracle.greedy_match(rp, ci, w)
    assert np.array_equal(got, _python_greedy(edges, 300, lambda c, a, b: (c, b, a)))
    assert np.array_equal(got, _python_greedy(edges, 300, lambda c, a, b: (c, a, b)))
    # the reverse tie-break (smaller endpoints first) is a different matching
    assert not np.array_equal(got, _python_greedy(edges, 300, lambda c, a, b: (c, -b, -a)))


def test_matching_poisson2d_closed_form():
    # all weights tie at 1.25; under the (c, b, a) order greedy pairs {2m, 2m+1} in every row
    m = 64
    rp, ci, val = P.poisson2d(m)
    w = oracle.edge_weights(rp, ci, val, np.ones(m * m))
    mate = oracle.greedy_match(rp, ci, w)
    idx = np.arange(m * m)
    assert np.array_equal(mate, idx ^ 1)


def test_matching_poisson3d_closed_form():
    m = 8
    rp, ci, val = P.poisson3d(m)
    w = oracle.edge_weights(rp, ci, val, np.ones(m ** 3))
    assert np.array_equal(oracle.greedy_match(rp, ci, w), np.arange(m ** 3) ^ 1)


def test_matching_is_maximal():
    rp, ci, val = P.random_spd(500, 5.0, seed=9)
    w = oracle.edge_weights(rp, ci, val, np.ones(500))
    mate = oracle.greedy_match(rp, ci, w)
    for (a, b) in _edges(rp, ci, w):
        assert mate[a] >= 0 or mate[b] >= 0


def test_matching_isolated_and_empty():
    # diagonal-only matrix: no edges, everything unmatched
    n = 5
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    w = oracle.edge_weights(rp, ci, np.full(n, 2.0), np.ones(n))
    assert np.all(oracle.greedy_match(rp, ci, w) == -1)
    assert np.all(oracle.suitor_match(rp, ci, w) == -1)

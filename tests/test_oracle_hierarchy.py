"""Pins of the oracle's hierarchy (Eq. Nmatrices and the +/- link rules, section "HEOM formalism").

The oracle sorts brute-force-enumerated tuples with a comparator and looks links up in a hash
table; these tests check it against the closed-form binomial counts (including the counts the paper
prints), the closed-form colexicographic rank, and a Python dictionary built independently.
"""
import itertools
import os
from math import comb

import numpy as np
import pytest

from oracle.oracle import hier_count, hier_export

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hierarchy_counts.txt")


def golden_counts():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        W, D, n, *_ = line.split()
        rows.append((int(W), int(D), int(n)))
    return rows


@pytest.mark.parametrize("M", range(1, 9))
@pytest.mark.parametrize("D", range(0, 7))
def test_count_is_binomial(M, D):
    assert hier_count(M, D) == comb(M + D, D)


@pytest.mark.parametrize("W,D,n", golden_counts())
def test_printed_counts(W, D, n):
    assert comb(W + D, W) == n
    assert hier_count(W, D) == n


def colex_index(t):
    """Closed form: level offset C(M+L-1, M) plus sum_j C(b_j, j) over bar positions b_j."""
    M = len(t)
    L = int(sum(t))
    off = comb(M + L - 1, M) if L > 0 else 0
    r, s = 0, 0
    for j in range(1, M):
        s += int(t[j - 1])
        r += comb((j - 1) + s, j)
    return off + r


@pytest.mark.parametrize("M,D", [(1, 5), (2, 4), (3, 3), (4, 4), (5, 3), (7, 2), (14, 4), (8, 6)])
def test_order_is_level_then_colex(M, D):
    t, _, _ = hier_export(M, D)
    idx = np.array([colex_index(row) for row in t])
    assert np.array_equal(idx, np.arange(len(t)))
    assert not np.any(t[0])  # root is the zero tuple


@pytest.mark.parametrize("M,D", [(1, 4), (2, 4), (3, 3), (4, 3), (5, 4), (6, 5), (8, 3)])
def test_links_against_dictionary(M, D):
    t, p, m = hier_export(M, D)
    pos = {tuple(int(x) for x in row): u for u, row in enumerate(t)}
    # every tuple with |n| <= D appears exactly once
    allt = [c for L in range(D + 1) for c in itertools.product(range(L + 1), repeat=M) if sum(c) == L]
    assert len(pos) == len(t) == len(allt) and set(pos) == set(allt)
    for u, row in enumerate(t):
        row = [int(x) for x in row]
        for l in range(M):
            up = row.copy(); up[l] += 1
            dn = row.copy(); dn[l] -= 1
            assert p[u, l] == (pos[tuple(up)] if sum(up) <= D else -1)
            assert m[u, l] == (pos[tuple(dn)] if dn[l] >= 0 else -1)


@pytest.mark.parametrize("M,D", [(14, 4), (10, 5)])
def test_link_invariants(M, D):
    t, p, m = hier_export(M, D)
    lev = t.sum(axis=1).astype(int)
    for l in range(M):
        ok = p[:, l] >= 0
        assert ok.sum() == comb(M + D - 1, M)           # all tuples below the top level
        assert np.all(m[p[ok, l], l] == np.nonzero(ok)[0])  # minus undoes plus
        assert np.all(lev[p[ok, l]] == lev[ok] + 1)
        okm = m[:, l] >= 0
        assert np.all(okm == (t[:, l] >= 1))
        assert np.all(p[m[okm, l], l] == np.nonzero(okm)[0])

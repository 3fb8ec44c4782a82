"""Pins for oracle.pattern: the index sets I(x_j) (eq:set_xj) and I(l) (eq:set_l)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import pattern
from workloads import iid_uniform, jittered


def brute_force_I_x(xj, Ms, m):
    """eq:set_xj by exhaustion over l and z, in exact rational arithmetic on u = fl(Ms x)."""
    u = Fraction(float(np.float64(Ms) * np.float64(xj)))
    out = []
    for l in range(-Ms // 2, Ms // 2):
        if any(-m <= u - l + Ms * z <= m for z in range(-3, 4)):
            out.append(l)
    return out


def brute_force_I_l(x, Ms, m):
    """eq:set_l by exhaustion over l, j and z."""
    cols = []
    for l in range(-Ms // 2, Ms // 2):
        col = []
        for j, xj in enumerate(x):
            u = Fraction(float(np.float64(Ms) * np.float64(xj)))
            if any(-m <= u - l + Ms * z <= m for z in range(-3, 4)):
                col.append(j)
        cols.append(col)
    return cols


def adversarial_nodes(Ms):
    """Grid points, their fp64 neighbours, the ends of the torus, and interior values."""
    xs = [-0.5, np.nextafter(0.5, 0.0), 0.0, np.nextafter(0.0, 1.0), -np.nextafter(0.0, 1.0)]
    for l in (-Ms // 2 + 1, -1, 1, Ms // 2 - 1):
        g = l / Ms
        xs += [g, np.nextafter(g, 1.0), np.nextafter(g, -1.0), g + 0.5 / Ms]
    return np.array(xs)


def test_golden_small_pattern(golden):
    for row in golden("pattern_Ms8_m1.txt"):
        got = pattern.index_sets_x(np.array([row[0]]), 8, 1)[0]
        assert list(got) == [int(v) for v in row[1:]]


@pytest.mark.parametrize("Ms,m", [(8, 1), (16, 3), (12, 2), (10, 4), (32, 4)])
def test_index_sets_x_brute_force(Ms, m):
    x = np.concatenate([adversarial_nodes(Ms), iid_uniform(Ms + m, 12)])
    got = pattern.index_sets_x(x, Ms, m)
    for j, xj in enumerate(x):
        assert list(got[j]) == brute_force_I_x(xj, Ms, m), (xj, Ms, m)


@pytest.mark.parametrize("Ms,m", [(8, 1), (16, 3), (10, 4)])
def test_index_sets_l_brute_force(Ms, m):
    x = np.concatenate([adversarial_nodes(Ms), jittered(5, 9)])
    want = brute_force_I_l(x, Ms, m)
    got = pattern.index_sets_l(x, Ms, m)
    assert [list(c) for c in got] == want
    ptr, idx = pattern.index_sets_l_fast(x, Ms, m)
    assert [list(idx[ptr[p]:ptr[p + 1]]) for p in range(Ms)] == want


def test_width_2m_or_2m_plus_1():
    """A node meets 2m+1 grid points iff M_sigma x_j is an integer, else 2m (2m < M_sigma)."""
    Ms, m = 64, 4
    x = np.concatenate([np.arange(-32, 32) / 64.0, iid_uniform(9, 200)])
    sets = pattern.index_sets_x(x, Ms, m)
    for xj, s in zip(x, sets):
        integer = float(Ms * xj).is_integer()
        assert len(s) == (2 * m + 1 if integer else 2 * m)


def test_nnz_identity():
    """sum_l |I(l)| = sum_j |I(x_j)| (the two views of one relation)."""
    x = iid_uniform(77, 300)
    Ms, m = 128, 6
    ptr, _ = pattern.index_sets_l_fast(x, Ms, m)
    assert ptr[-1] == sum(len(s) for s in pattern.index_sets_x(x, Ms, m))

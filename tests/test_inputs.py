"""Input generators: the Halton sequence against hand-derived values (the
paper's point sets, Sec. 6.2) and the SplitMix64 stream's determinism."""
from fractions import Fraction

import numpy as np

from conftest import read_golden
from paper_1708_09707_gb300 import inputs


def test_halton_matches_hand_derived_values():
    rows = read_golden("halton.txt")
    P = inputs.halton_points(len(rows), 3)
    for k, row in enumerate(rows):
        assert int(row[0]) == k + 1
        for dim in range(3):
            assert P[k, dim] == float(Fraction(row[1 + dim])), (k, dim)


def test_halton_start_offset_and_range():
    a = inputs.halton_points(100, 2)
    b = inputs.halton_points(90, 2, start=11)
    assert np.array_equal(a[10:], b)
    assert a.min() > 0.0 and a.max() < 1.0
    # base 2 coordinates of 1 .. 2^k - 1 are exactly the odd multiples of
    # 2^-j, j <= k: a permutation of i / 2^k, i = 1 .. 2^k - 1
    k = 10
    h = np.sort(inputs.halton_points((1 << k) - 1, 1)[:, 0])
    assert np.array_equal(h, np.arange(1, 1 << k) / float(1 << k))


def test_splitmix_stream_is_counter_based():
    g = inputs.SplitMix64(77)
    a = g.u64(5)
    b = g.u64(3)
    c = inputs.SplitMix64(77).u64(8)
    assert np.array_equal(np.concatenate([a, b]), c)

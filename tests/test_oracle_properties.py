"""Property tests of the oracle's block structure (Alg. 1 with the
admissibility condition of Sec. 2.3) over random sizes, dimensions, leaf
sizes, eta, both admissibility forms and point sets with exact duplicates,
for one set and for two sets:
  - the leaves tile I x I (I1 x I2) exactly once;
  - every admissible leaf satisfies the condition, recomputed here from the
    boxes with numpy;
  - every dense leaf has a side of at most C_leaf: Alg. 1 splits every
    inadmissible pair whose sides both exceed C_leaf;
  - eta = 0 admits no pair of clusters with positive diameters."""
import numpy as np
import pytest

from paper_1708_09707_gb300 import inputs

try:
    from hypothesis import given, settings, strategies as st
    HAVE_HYPOTHESIS = True
except ImportError:   # a machine without hypothesis draws the cases with numpy
    HAVE_HYPOTHESIS = False


def _points(n, d, seed, dup):
    p = inputs.uniform_points(n, d, seed)
    if dup:
        p = np.round(p * 4.0) / 4.0      # a coarse grid: many exact duplicates
    return p


def _check(H, n1, n2, leaf, eta, adm_max, rect):
    lo, hi, bmin, bmax = H.tree()
    if rect:
        lo2, hi2, bmin2, bmax2 = H.col_tree()
    else:
        lo2, hi2, bmin2, bmax2 = lo, hi, bmin, bmax
    cover = np.zeros((n1, n2), np.int32)
    for t, s in H.adm_leaves():
        cover[lo[t]:hi[t], lo2[s]:hi2[s]] += 1
        dt = np.sum((bmax[t] - bmin[t]) ** 2)
        ds = np.sum((bmax2[s] - bmin2[s]) ** 2)
        g = (np.maximum(0, bmin[t] - bmax2[s]) ** 2 + np.maximum(0, bmin2[s] - bmax[t]) ** 2).sum()
        diam = max(dt, ds) if adm_max else min(dt, ds)
        assert diam <= eta * eta * g * (1 + 1e-12) + 1e-300
        if eta == 0.0:
            assert diam == 0.0
    for t, s in H.dense_leaves():
        cover[lo[t]:hi[t], lo2[s]:hi2[s]] += 1
        assert min(hi[t] - lo[t], hi2[s] - lo2[s]) <= leaf
    assert (cover == 1).all()


def _one_set(orc, n, d, leaf, eta, adm_max, dup, seed):
    pts = _points(n, d, seed, dup)
    H = orc.HMatrix(pts, 0, 0.2, leaf, eta, 1e-6, adm_max=adm_max, compress=False)
    _check(H, n, n, leaf, eta, adm_max, False)


def _two_sets(orc, n1, n2, d, leaf, eta, dup, seed):
    P = _points(n1, d, seed, dup)
    Q = _points(n2, d, seed + 1, dup)
    H = orc.HMatrix(P, 0, 0.2, leaf, eta, 1e-6, compress=False, cols=Q)
    _check(H, n1, n2, leaf, eta, False, True)


if HAVE_HYPOTHESIS:
    @settings(max_examples=40, deadline=None)
    @given(n=st.integers(1, 400), d=st.integers(1, 3), leaf=st.integers(1, 48),
           eta=st.sampled_from([0.0, 0.5, 1.0, 1.5, 2.0]), adm_max=st.booleans(),
           dup=st.booleans(), seed=st.integers(0, 10_000))
    def test_block_structure_one_set(orc, n, d, leaf, eta, adm_max, dup, seed):
        _one_set(orc, n, d, leaf, eta, adm_max, dup, seed)

    @settings(max_examples=30, deadline=None)
    @given(n1=st.integers(1, 300), n2=st.integers(1, 300), d=st.integers(1, 3),
           leaf=st.integers(1, 40), eta=st.sampled_from([0.0, 1.0, 1.5]), dup=st.booleans(),
           seed=st.integers(0, 10_000))
    def test_block_structure_two_sets(orc, n1, n2, d, leaf, eta, dup, seed):
        _two_sets(orc, n1, n2, d, leaf, eta, dup, seed)
else:
    def test_block_structure_one_set(orc):
        rng = np.random.default_rng(20260)
        for _ in range(40):
            _one_set(orc, int(rng.integers(1, 401)), int(rng.integers(1, 4)),
                     int(rng.integers(1, 49)), float(rng.choice([0.0, 0.5, 1.0, 1.5, 2.0])),
                     bool(rng.integers(2)), bool(rng.integers(2)), int(rng.integers(10_001)))

    def test_block_structure_two_sets(orc):
        rng = np.random.default_rng(20261)
        for _ in range(30):
            _two_sets(orc, int(rng.integers(1, 301)), int(rng.integers(1, 301)),
                      int(rng.integers(1, 4)), int(rng.integers(1, 41)),
                      float(rng.choice([0.0, 1.0, 1.5])), bool(rng.integers(2)),
                      int(rng.integers(10_001)))

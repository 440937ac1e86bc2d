"""Pins of the oracle's structure steps (Morton codes, sort, cluster tree,
bounding boxes, admissibility, Alg. 1 leaf partition)."""
import functools

import numpy as np
import pytest

from conftest import read_golden
from paper_1708_09707_gb300 import inputs


def test_morton_hand_derived(orc):
    rows = read_golden("morton_codes.txt")
    groups = {}
    for d, coords, code in rows:
        groups.setdefault(int(d), []).append(
            ([float(c) for c in coords.split()], int(code, 16)))
    for d, items in groups.items():
        pts = np.array([c for c, _ in items])
        codes, bits, lo, hi, _ = orc.morton(pts)
        assert bits == min(32, 64 // d)
        assert [int(c) for c in codes] == [c for _, c in items], d


def _zorder_cmp(a, b, k, d):
    # Recursive quadrant/octant order on the 2^k grid: at each level from the
    # top, the cell index is sum_i bit(x_i) * 2^(d-1-i); the first level
    # where the cells differ decides.
    for lev in range(k - 1, -1, -1):
        ca = sum(((a[i] >> lev) & 1) << (d - 1 - i) for i in range(d))
        cb = sum(((b[i] >> lev) & 1) << (d - 1 - i) for i in range(d))
        if ca != cb:
            return -1 if ca < cb else 1
    return 0


@pytest.mark.parametrize("d,k", [(2, 4), (3, 3), (1, 6)])
def test_morton_order_is_recursive_z_order(orc, d, k):
    side = 1 << k
    grid = np.stack(np.meshgrid(*[np.arange(side)] * d, indexing="ij"), -1)
    grid = grid.reshape(-1, d)
    rng = np.random.default_rng(d)
    grid = grid[rng.permutation(len(grid))]
    # coordinates (g + 0.5) / side in a box fixed to [0,1] by two corner points
    pts = np.vstack([(grid + 0.5) / side, np.zeros((1, d)), np.ones((1, d))])
    codes, *_ = orc.morton(pts)
    perm = orc.sort(codes)
    perm = perm[(perm < len(grid))]
    cells = [tuple(int(v) for v in grid[p]) for p in perm]
    ref = sorted((tuple(int(v) for v in g) for g in grid),
                 key=functools.cmp_to_key(lambda a, b: _zorder_cmp(a, b, k, d)))
    assert cells == ref


def test_sort_matches_numpy_stable(orc):
    rng = np.random.default_rng(1)
    codes = rng.integers(0, 50, size=5000).astype(np.uint64)  # many ties
    perm = orc.sort(codes)
    assert np.array_equal(perm, np.argsort(codes, kind="stable"))


def test_morton_degenerate_dimension(orc):
    # all points share y: scale 0 in that dimension, its bits stay 0
    pts = np.array([[0.0, 0.3], [1.0, 0.3], [0.5, 0.3]])
    codes, _, lo, hi, sc = orc.morton(pts)
    assert sc[1] == 0.0
    assert codes[0] == 0 and codes[2] == 1 << 63


@pytest.mark.parametrize("n,leaf", [(1, 1), (2, 1), (7, 2), (64, 64), (65, 64),
                                    (129, 64), (1000, 32), (4096, 32),
                                    (100003, 64)])
def test_tree_halving_closed_form(orc, n, leaf):
    lo, hi = orc.tree_ranges(n, leaf)
    depth = orc.tree_depth(n, leaf)
    # depth: smallest l with ceil(n / 2^l) <= leaf
    l = 0
    while -(-n // (1 << l)) > leaf:
        l += 1
    assert depth == l
    present = lo >= 0
    for v in np.nonzero(present)[0]:
        lev = int(np.floor(np.log2(v + 1)))
        size = hi[v] - lo[v]
        assert size in (n >> lev, -(-n // (1 << lev))) or lev == 0
        internal = size > leaf
        c1, c2 = 2 * v + 1, 2 * v + 2
        if internal:
            assert lo[c1] == lo[v] and hi[c1] == lo[v] + size // 2
            assert lo[c2] == hi[c1] and hi[c2] == hi[v]
        elif c1 < lo.size:
            assert lo[c1] < 0 and lo[c2] < 0
    leaves = [v for v in np.nonzero(present)[0]
              if hi[v] - lo[v] <= leaf]
    cover = np.zeros(n, np.int64)
    for v in leaves:
        cover[lo[v]:hi[v]] += 1
    assert np.all(cover == 1)
    assert np.all(hi[leaves] - lo[leaves] >= 1)


def test_bbox_matches_numpy(orc):
    pts = inputs.uniform_points(3000, 3, 7)
    lo, hi, bmin, bmax = orc.bbox(pts, 40)
    for v in range(lo.size):
        if lo[v] < 0:
            continue
        seg = pts[lo[v]:hi[v]]
        assert np.array_equal(bmin[v], seg.min(0))
        assert np.array_equal(bmax[v], seg.max(0))


def test_admissibility_hand_boxes(orc):
    for form, eta, tmin, tmax, smin, smax, exp in read_golden("admissibility.txt"):
        f = lambda s: np.array([float(v) for v in s.split()])
        got = orc.admissible(f(tmin), f(tmax), f(smin), f(smax), float(eta),
                             use_max=(form == "max"))
        assert got == bool(int(exp)), (form, eta, tmin, tmax, smin, smax)
        # the relation is symmetric in (tau, sigma)
        assert orc.admissible(f(smin), f(smax), f(tmin), f(tmax), float(eta),
                              use_max=(form == "max")) == got


def _leaves_str(arr):
    return " ".join("%d:%d" % (t, s) for t, s in arr)


def test_block_tree_hand_1d(orc):
    x = np.array([5, 2, 7, 0, 3, 6, 1, 4], dtype=np.float64)[:, None]
    for eta, adm, dense in read_golden("blocktree_1d.txt"):
        h = orc.HMatrix(x, 0, 1.0, 2, float(eta), 1e-8, compress=False)
        assert np.array_equal(h.perm(), [3, 6, 1, 4, 7, 0, 5, 2])
        assert _leaves_str(h.adm_leaves()) == adm, eta
        assert _leaves_str(h.dense_leaves()) == dense, eta


def check_partition(h, n, leaf, eta, adm_max=False, orc=None):
    """Invariants of Alg. 1's leaf set, checked by brute force."""
    lo, hi, bmin, bmax = h.tree()
    cover = np.zeros((n, n), np.int32)
    A, D = h.adm_leaves(), h.dense_leaves()
    for t, s in A:
        cover[lo[t]:hi[t], lo[s]:hi[s]] += 1
        assert orc.admissible(bmin[t], bmax[t], bmin[s], bmax[s], eta, adm_max)
    for t, s in D:
        cover[lo[t]:hi[t], lo[s]:hi[s]] += 1
        assert not orc.admissible(bmin[t], bmax[t], bmin[s], bmax[s], eta, adm_max)
        assert min(hi[t] - lo[t], hi[s] - lo[s]) <= leaf
        assert max(hi[t] - lo[t], hi[s] - lo[s]) <= leaf + 1
    assert np.all(cover == 1)
    # every internal block node (an ancestor pair of a leaf) is inadmissible
    # with both sides > leaf: walk up from each leaf
    for t, s in np.vstack([A, D]):
        while t > 0:
            t, s = (t - 1) // 2, (s - 1) // 2
            assert hi[t] - lo[t] > leaf and hi[s] - lo[s] > leaf
            assert not orc.admissible(bmin[t], bmax[t], bmin[s], bmax[s], eta, adm_max)
    # canonical order
    keys = [(lo[t], lo[s]) for t, s in A]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)


@pytest.mark.parametrize("n,d,leaf,eta,adm_max,kind", [
    (1, 2, 4, 1.0, False, "uniform"),
    (5, 2, 4, 1.0, False, "uniform"),
    (777, 2, 16, 1.0, True, "uniform"),
    (1024, 3, 8, 1.0, False, "uniform"),
    (1500, 2, 33, 1.5, False, "mixture"),
    (600, 1, 7, 0.7, False, "uniform"),
])
def test_block_tree_partition_invariants(orc, n, d, leaf, eta, adm_max, kind):
    pts = (inputs.uniform_points(n, d, 11) if kind == "uniform"
           else inputs.mixture_points(n, d, 11))
    h = orc.HMatrix(pts, 0, 0.1, leaf, eta, 1e-6, adm_max=adm_max, compress=False)
    check_partition(h, n, leaf, eta, adm_max, orc)


def test_block_tree_all_points_equal(orc):
    # zero-diameter clusters: every off-diagonal... every pair has min diam 0
    # and dist 0, so 0 <= 0 makes the root itself admissible
    pts = np.full((300, 2), 0.25)
    h = orc.HMatrix(pts, 0, 0.1, 8, 1.0, 1e-6, compress=False)
    assert h.n_adm == 1 and h.n_dense == 0
    lo, hi, _, _ = h.tree()
    assert tuple(h.adm_leaves()[0]) == (0, 0)

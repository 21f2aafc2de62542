"""Pins of the oracle's voxel maps (Sec. III-C, Eq. (10)) and score (Eq. (11)):
special cases with known keys, the set definition, a planted voxel-centre scan
built with an independent rotation library, and the upper-bound property."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2310_10023_gb300 import synth


def _keyset(a):
    return set(map(tuple, np.asarray(a).reshape(-1, 3).tolist()))


def test_voxel_centre_keys():
    # points at voxel centres (v + 1/2) r have key v at level 0 and floor(v / 2^l) above
    r = 0.25
    v = np.array([[0, 0, 0], [-1, -1, -1], [5, -7, 3], [-100, 40, 0]], np.int64)
    pts = ((v + 0.5) * r).astype(np.float32)
    M = oracle.Maps(pts, r, 3, oracle.LEAF_UNDILATED)
    assert _keyset(M.keys(0)) == _keyset(v)
    for l in (1, 2):
        base = np.floor_divide(v, 2 ** l)
        want = {tuple(b - np.array(j)) for b in base for j in np.ndindex(2, 2, 2)}
        assert _keyset(M.keys(l)) == want


def test_negative_coordinates_floor():
    M = oracle.Maps(np.array([[-0.1, 0.1, -0.6]], np.float32), 0.5, 1, oracle.LEAF_UNDILATED)
    assert _keyset(M.keys(0)) == {(-1, 0, -2)}


def test_single_point_dilation():
    # one occupied voxel: every level stores the 8 voxels v - j, j in {0,1}^3
    M = oracle.Maps(np.array([[3.3, -2.2, 0.7]], np.float32), 1.0, 4)
    for l in range(4):
        v = np.floor_divide(np.array([3, -3, 0]), 2 ** l)
        assert _keyset(M.keys(l)) == {tuple(v - np.array(j)) for j in np.ndindex(2, 2, 2)}


def test_maps_match_set_definition(room):
    w, m, _, _ = room
    M = oracle.Maps(m, w.r, w.levels)
    rho = np.float32(1.0 / float(np.float32(w.r)))
    u = np.floor(m.astype(np.float32) * rho).astype(np.int64)   # FP32 product, one rounding
    u = np.unique(u, axis=0)
    for l in range(w.levels):
        b = np.unique(np.floor_divide(u, 2 ** l), axis=0)
        d = np.unique(np.concatenate([b - np.array(j) for j in np.ndindex(2, 2, 2)]), axis=0)
        assert _keyset(M.keys(l)) == _keyset(d)
        # hash table: T_l > count and every stored key is found, a shifted one is not
        assert M.table_size(l) > M.count(l)
    M2 = oracle.Maps(m, w.r, w.levels, oracle.LEAF_UNDILATED)
    assert _keyset(M2.keys(0)) == _keyset(u)


def test_map_contains_is_membership():
    rng = np.random.default_rng(1)
    pts = rng.uniform(-5, 5, size=(2000, 3)).astype(np.float32)
    M = oracle.Maps(pts, 0.5, 2)
    ks = _keyset(M.keys(1))
    for _ in range(3000):
        q = tuple(int(x) for x in rng.integers(-8, 8, 3))
        assert M.contains(1, q) == (q in ks)


def test_map_errors():
    with pytest.raises(ValueError):
        oracle.Maps(np.array([[np.nan, 0, 0]], np.float32), 0.5, 2)
    with pytest.raises(ValueError):
        oracle.Maps(np.zeros((1, 3), np.float32), 0.0, 2)
    with pytest.raises(ValueError):
        oracle.Maps(np.array([[3e6, 0, 0]], np.float32), 1.0, 2)   # key beyond 2^20
    M = oracle.Maps(np.zeros((0, 3), np.float32), 0.5, 2)
    assert M.count(0) == 0


# --------------------------------------------------------------------------
# Eq. (11) score
# --------------------------------------------------------------------------

def _planted(grid_r=0.5, levels=3, seed=0, k=300):
    """Scan = voxel centres of an occupied set seen from a grid-exact leaf pose,
    inverse-transformed with scipy; every point must hit at that leaf."""
    rng = np.random.default_rng(seed)
    m, _ = synth.make_map(1), None
    rg = oracle.make_ranges((0, 0, 0), (20, 20, 5), (-0.05, -0.05, 0.0), (0.05, 0.05, 2 * math.pi))
    g = oracle.Grid(grid_r, levels, 20.0, rg)
    M = oracle.Maps(m, grid_r, levels, oracle.LEAF_UNDILATED)
    keys = M.keys(0)
    sel = keys[rng.choice(len(keys), size=k, replace=False)]
    r = float(np.float32(grid_r))
    centres = (sel.astype(np.float64) + 0.5) * r
    T = np.array([int(rng.integers(5, 30)), int(rng.integers(5, 30)), int(rng.integers(0, 6))])
    ia, ib, ig = (int(rng.integers(0, g.N(0)[i])) for i in range(3))
    R = Rotation.from_euler("ZYX", [g.angle(0, 2, ig), g.angle(0, 1, ib), g.angle(0, 0, ia)]).as_matrix()
    scan = ((centres - T * r) @ R).astype(np.float32)          # s = R^T (p - t)
    leaf = [int(T[0]), int(T[1]), int(T[2]), ia, ib, ig, 0]
    return M, g, scan, leaf, sel


@pytest.mark.parametrize("seed", range(3))
def test_planted_voxel_centres_score_k(seed):
    M, g, scan, leaf, _ = _planted(seed=seed)
    assert M.score_nodes(g, scan, [leaf])[0] == len(scan)
    # a shifted translation loses points
    moved = list(leaf)
    moved[0] += 3
    assert M.score_nodes(g, scan, [moved])[0] < len(scan)


def test_score_matches_set_lookup(room):
    """Score = number of points whose level key is in the level's set (Eq. (11)),
    recomputed point by point with a Python set."""
    w, m, s, _ = room
    M = oracle.Maps(m, w.r, w.levels)
    rg = oracle.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), rg)
    rng = np.random.default_rng(5)
    sets = [_keyset(M.keys(l)) for l in range(w.levels)]
    for _ in range(40):
        l = int(rng.integers(0, w.levels))
        node = [int(rng.integers(0, 40 >> l)), int(rng.integers(0, 40 >> l)), int(rng.integers(0, 10 >> l)),
                int(rng.integers(0, g.N(l)[0])), int(rng.integers(0, g.N(l)[1])), int(rng.integers(0, g.N(l)[2])), l]
        A = g.rotation(l, *node[3:6]).reshape(3, 3)
        # FP32 products and sums in the fixed order, one rounding each
        p = [A[i, 0] * s[:, 0] for i in range(3)]
        q = np.stack([(A[i, 0] * s[:, 0] + A[i, 1] * s[:, 1]).astype(np.float32) + A[i, 2] * s[:, 2]
                      for i in range(3)], 1).astype(np.float32)
        del p
        u = np.floor(q).astype(np.int64) + np.array(node[:3]) * 2 ** l
        keys = np.floor_divide(u, 2 ** l)
        want = sum(tuple(k) in sets[l] for k in keys.tolist())
        assert M.score_nodes(g, s, [node])[0] == want


def test_translation_only_upper_bound(room):
    """With translation-only branching the dilated parent's score bounds every
    child's (the property the dilation of Sec. III-C is for)."""
    w, m, s, _ = room
    M = oracle.Maps(m, w.r, w.levels)
    rg = oracle.make_ranges(w.lo, w.hi, (-0.03, -0.03, 0.0), (0.03, 0.03, 2 * math.pi))
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), rg, oracle.TRANSLATION_ONLY)
    rng = np.random.default_rng(7)
    for _ in range(60):
        l = int(rng.integers(1, w.levels))
        p = [int(rng.integers(-2, 42 >> l)), int(rng.integers(-2, 42 >> l)), int(rng.integers(-1, 11 >> l)),
             int(rng.integers(0, g.N(l)[0])), int(rng.integers(0, g.N(l)[1])), int(rng.integers(0, g.N(l)[2])), l]
        ps = M.score_nodes(g, s, [p])[0]
        kids = g.children(p)
        ks = M.score_nodes(g, s, kids)
        assert ks.max() <= ps


def test_score_rejects_invalid_nodes(room):
    w, m, s, _ = room
    M = oracle.Maps(m, w.r, w.levels)
    rg = oracle.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), rg)
    for bad in ([0, 0, 0, 0, 0, 0, 3], [0, 0, 0, -1, 0, 0, 0], [0, 0, 0, 0, 0, g.N(1)[2], 1],
                [1 << 21, 0, 0, 0, 0, 0, 0]):
        with pytest.raises(ValueError):
            M.score_nodes(g, s, [bad])

"""Pins of the oracle's exact-bound dilation (orc_exact_dilation; the
remedy for the approximate rotational bound of Sec. III-D).

A level-l node's score bounds the scores of all its leaves when the level-l
map is widened far enough: a leaf hit at fine key k_d = u_d + c 2^l + t
(t in [0, 2^l) per axis, the leaf below translation c; the leaf map holds
b - j0, j0 in {0, 1}) has b >> l = ((u_d + t + j0) >> l) + c, while the node
probes (u_p >> l) + c.  So the widening E must cover, per axis,
(u_d >> l) - (u_p >> l) >= -E and ((u_d + 2^l) >> l) - (u_p >> l) <= 1 + E,
where u_p and u_d are the FP32 fine keys of a scan point under the node's and
the leaf's rotations.  The tests measure that requirement directly -- every
(node, leaf) rotation pair of the grid, points on a sphere at the scan's
reach -- and check the oracle's derived e against it; they check the
score-level invariant (node score >= every leaf's) on the room map with exact
maps, show it failing without the widening, and build a one-point case where
a widening one below the measured requirement loses a leaf hit that the
oracle's e keeps.

The derived e has slack (it sums the three axes' half-segment angles and
allows 2 voxels for the floors and FP32 rounding): on these grids the
measured requirement is 1 to 5 while e is 2 to 13.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2310_10023_gb300 import synth

RP = 0.0523599      # roll / pitch half range, 3 degrees


def _sphere(n, radius):
    """n points spread evenly on a sphere (Fibonacci lattice), FP32."""
    i = np.arange(n) + 0.5
    phi = np.arccos(1 - 2 * i / n)
    th = math.pi * (1 + 5 ** 0.5) * i
    return (radius * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)).astype(np.float32)


def _keys(table, pts):
    """Fine keys floor((A_i0 x + A_i1 y) + A_i2 z), every product and sum in
    FP32 (numpy float32: one rounding per operation, no FMA): (n_rot, 3, n_pts)."""
    A = table.astype(np.float32).reshape(-1, 3, 3)
    x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
    q = (A[:, :, None, 0] * x + A[:, :, None, 1] * y) + A[:, :, None, 2] * z
    assert q.dtype == np.float32
    return np.floor(q).astype(np.int64)


def _leaf_rotations(g, l, rot):
    """Level-0 rotation indices below rotation `rot` of level l (Eq. (13)
    children of the oracle, followed down to the leaves)."""
    na, nb, ng = g.N(l)
    nodes = [(0, 0, 0, rot // (nb * ng), (rot // ng) % nb, rot % ng, l)]
    for _ in range(l):
        nodes = [tuple(c) for nd in nodes for c in g.children(np.array(nd, np.int32)) if c[0] == c[1] == c[2] == 0]
    _, nb0, ng0 = g.N(0)
    return sorted({(c[3] * nb0 + c[4]) * ng0 + c[5] for c in nodes})


def _requirement(g, pts):
    """Per level, the widening every (node, leaf, point, axis) needs, and one
    pair that needs it: (E, (rot_node, rot_leaf, point, axis, t_high))."""
    U0 = _keys(g.rotation_table(0), pts)
    out = {}
    for l in range(1, g.levels):
        Ul = _keys(g.rotation_table(l), pts)
        best, arg = -1, None
        for r in range(len(Ul)):
            lv = _leaf_rotations(g, l, r)
            lo = (U0[lv] >> l) - (Ul[r][None] >> l)                 # t = 0, j0 = 0
            hi = ((U0[lv] + (1 << l)) >> l) - (Ul[r][None] >> l)    # t + j0 = 2^l
            need = np.maximum(-lo, hi - 1)
            i = np.unravel_index(int(np.argmax(need)), need.shape)
            if need[i] > best:
                best = int(need[i])
                arg = (r, lv[i[0]], i[2], i[1], bool(hi[i] - 1 >= -lo[i]))
        out[l] = (best, arg)
    return out


def _grid(w, grid_dmax, rp=RP, flags=0):
    rg = oracle.make_ranges(w.lo, w.hi, (-rp, -rp, 0.0), (rp, rp, 2 * math.pi))
    return oracle.Grid(w.r, w.levels, grid_dmax, rg, flags)


CASES = [
    # (grid d_max, roll/pitch half range, flags): the default reading with
    # the scan's own reach; yaw only with a grid d_max well below the reach;
    # the lower-edge reading (whole segments) with a short grid d_max
    (None, RP, 0),
    (6.0, 0.0, 0),
    (3.0, RP, 0),
    (12.0, RP, oracle.ANGLE_LOWER_EDGE),
]


@pytest.mark.parametrize("grid_dmax,rp,flags", CASES)
def test_derived_dilation_covers_the_measured_requirement(room, grid_dmax, rp, flags):
    w, _, s, _ = room
    reach = oracle.scan_dmax(s)
    g = _grid(w, grid_dmax or reach, rp, flags)
    e = g.exact_dilation(reach)
    pts = np.concatenate([_sphere(200, reach * (1 - 1e-6)), s[np.argsort(-np.linalg.norm(s, axis=1))[:40]]])
    req = _requirement(g, pts)
    need = max(v[0] for v in req.values())
    assert need >= 1                 # the approximate bound (no widening) does not hold
    assert e >= need, (e, req)       # the derived widening covers every pair measured
    # the requirement grows with the reach beyond the grid's d_max, and so does e
    if grid_dmax is not None and grid_dmax < reach / 2:
        assert need >= 2 and e > g.exact_dilation(grid_dmax)


def test_node_scores_bound_leaf_scores_with_exact_maps(room):
    """Score-level invariant on the room map (full yaw, roll/pitch 3 degrees):
    500 random nodes per level above the leaves, every leaf below each of
    them scored with the scan's 200 farthest points (at d_max, where rotation
    moves a point most) and 200 others; with the oracle's e no leaf beats its
    node.  (Random nodes rarely catch the approximate bound failing; the gap
    test below does.)"""
    w, m, s, _ = room
    order = np.argsort(-np.linalg.norm(s, axis=1))
    s = np.ascontiguousarray(np.concatenate([s[order[:200]], s[order[200::4][:200]]]))
    rg = oracle.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    dm = oracle.scan_dmax(s)
    g = oracle.Grid(w.r, w.levels, dm, rg)
    e = g.exact_dilation(dm)
    rng = np.random.default_rng(0)
    (a0, a1, a2), (b0, b1, b2) = g.wrange()
    parents = {}
    for l in range(1, w.levels):
        sh = w.levels - 1 - l
        parents[l] = np.array([[int(rng.integers(a0 << sh, (b0 + 1) << sh)), int(rng.integers(a1 << sh, (b1 + 1) << sh)),
                                int(rng.integers(a2 << sh, (b2 + 1) << sh)),
                                *(int(rng.integers(0, g.N(l)[i])) for i in range(3)), l] for _ in range(500)], np.int32)

    def leaves(p):
        nodes = [p]
        for _ in range(int(p[6])):
            nodes = [c for nd in nodes for c in g.children(nd)]
        return np.array(nodes, np.int32)

    below = {l: [leaves(p) for p in parents[l]] for l in parents}
    M = oracle.Maps(m, w.r, w.levels, oracle.exact_flags(e))
    checked = 0
    for l in parents:
        ps = M.score_nodes(g, s, parents[l])
        ls = M.score_nodes(g, s, np.concatenate(below[l]))
        off = 0
        for i, lv in enumerate(below[l]):
            assert (ls[off:off + len(lv)] <= ps[i]).all(), (l, parents[l][i])
            off += len(lv)
            checked += len(lv)
    assert checked > 10000


def _ancestor(g, leaf, l):
    """The level-l node above a leaf: translation floor(c / 2^l), and per
    axis the level-l segment among whose Eq. (13) children the leaf's lies."""
    node = [int(leaf[i]) >> l for i in range(3)]
    rot = [int(leaf[3 + i]) for i in range(3)]
    for lv in range(1, l + 1):
        N = g.N(lv)
        up = []
        for i in range(3):
            cands = [c for c in range(max(0, rot[i] // 2 - 3), min(N[i], rot[i] // 2 + 4))
                     if rot[i] in _axis_children(g, lv, i, c, N)]
            assert len(cands) == 1
            up.append(cands[0])
        rot = up
    return np.array([*node, *rot, l], np.int32)


def _axis_children(g, lv, axis, c, N):
    nd = [0, 0, 0, 0, 0, 0, lv]
    nd[3 + axis] = c
    for j in range(3):
        if j != axis:
            nd[3 + j] = 0
    kids = g.children(np.array(nd, np.int32))
    return {int(k[3 + axis]) for k in kids}


def test_exact_bound_closes_the_gap_of_the_approximate_bound(room):
    """A room window (scan 1, yaw +-0.3 rad around the planted yaw, 6 x 6 x 2 m)
    where the approximate bound misses the optimum: its BnB returns 999 of
    1000 points while the exhaustive maximum over the same leaves is 1000.
    The best leaf's ancestors explain it: some score below the leaf under the
    plain maps.  With the exact-bound maps every ancestor scores at least the
    leaf and the BnB returns the exhaustive maximum."""
    w, m, _, _ = room
    s, pose = synth.make_scan(w.scene, 1)
    x0 = math.floor(pose[0] / 2.0) * 2.0 - 2.0
    y0 = math.floor(pose[1] / 2.0) * 2.0 - 2.0
    rg = oracle.make_ranges((x0, y0, 0.0), (x0 + 5.9, y0 + 5.9, 1.9), (-RP, -RP, pose[5] - 0.3),
                            (RP, RP, pose[5] + 0.3))
    dm = oracle.scan_dmax(s)
    g = oracle.Grid(w.r, w.levels, dm, rg)
    M = oracle.Maps(m, w.r, w.levels)
    best, leaf = oracle.brute_force(M, g, s)
    approx = oracle.localize(M, s, rg, score_frac=0.95, batch=w.batch)
    assert approx.status == oracle.OK and approx.best_score < best
    anc = np.array([_ancestor(g, leaf, l) for l in range(1, w.levels)])
    assert (M.score_nodes(g, s, anc) < best).any()
    e = g.exact_dilation(dm)
    ME = oracle.Maps(m, w.r, w.levels, oracle.exact_flags(e))
    assert (ME.score_nodes(g, s, anc) >= best).all()
    assert ME.score_nodes(g, s, [list(leaf)])[0] == best
    exact = oracle.localize(ME, s, rg, score_frac=0.95, batch=w.batch)
    assert exact.status == oracle.OK and exact.best_score == best


@pytest.mark.parametrize("grid_dmax,rp,flags", CASES[1:3])
def test_one_below_the_requirement_loses_a_leaf_hit(room, grid_dmax, rp, flags):
    """One scan point and a one-voxel map, placed at the pair that needs the
    largest widening: the leaf scores 1; its level-l ancestor scores 1 with
    the oracle's e and 0 with a widening one below the measured requirement,
    so the node would no longer bound its leaf."""
    w, _, s, _ = room
    reach = oracle.scan_dmax(s)
    g = _grid(w, grid_dmax, rp, flags)
    pts = _sphere(200, reach * (1 - 1e-6))
    req = _requirement(g, pts)
    l = max(req, key=lambda k: req[k][0])
    need, (rn, rd, ip, axis, high) = req[l]
    assert need >= 2
    e = g.exact_dilation(reach)
    p = pts[ip:ip + 1]
    _, nb0, ng0 = g.N(0)
    _, nbl, ngl = g.N(l)
    ud = _keys(g.rotation_table(0)[rd:rd + 1], p)[0, :, 0]
    # the node's translation and the leaf's offset below it: on the worst axis
    # the offset that needs the widening, elsewhere 0
    cp = np.array([3, -2, 1], np.int64)
    t = np.zeros(3, np.int64)
    if high:
        t[axis] = (1 << l) - 1
    T = cp * (1 << l) + t
    b = ud + T + (1 if high else 0) * (np.arange(3) == axis)   # the leaf's hit (j0 = 1 on a high axis)
    mp = ((b.astype(np.float64) + 0.5) * w.r).astype(np.float32)[None]   # the voxel's centre
    leaf = [*T.tolist(), rd // (nb0 * ng0), (rd // ng0) % nb0, rd % ng0, 0]
    node = [*cp.tolist(), rn // (nbl * ngl), (rn // ngl) % nbl, rn % ngl, l]
    full = oracle.Maps(mp, w.r, w.levels, oracle.exact_flags(e))
    short = oracle.Maps(mp, w.r, w.levels, oracle.exact_flags(need - 1) if need > 1 else 0)
    assert full.contains(0, b)
    assert full.score_nodes(g, p, [leaf])[0] == 1
    assert short.score_nodes(g, p, [leaf])[0] == 1
    assert full.score_nodes(g, p, [node])[0] == 1
    assert short.score_nodes(g, p, [node])[0] == 0

"""Pins of the oracle's depth-first batched order (Table I's DFS search
strategy): every kept node scores above best, so where the bound is exact the
result's score is the exhaustive optimum -- the same as the best-first
order's -- however the nodes are ordered."""
import math

import pytest

import oracle
from paper_2310_10023_gb300 import synth


def _window_ranges(pose, half_yaw=0.12, rp=0.02):
    x0 = math.floor(pose[0] / 2.0) * 2.0 - 2.0
    y0 = math.floor(pose[1] / 2.0) * 2.0 - 2.0
    return oracle.make_ranges((x0, y0, 0.0), (x0 + 3.9, y0 + 3.9, 1.9),
                              (-rp, -rp, pose[5] - half_yaw), (rp, rp, pose[5] + half_yaw))


@pytest.mark.parametrize("scan_index", [0, 1])
@pytest.mark.parametrize("batch", [1, 64, 100000])
def test_dfs_translation_only_equals_brute_force(room, scan_index, batch):
    w, m, _, _ = room
    s, pose = synth.make_scan(1, scan_index)
    s = s[:200]
    M = oracle.Maps(m, w.r, w.levels)
    rg = _window_ranges(pose)
    flags = oracle.TRANSLATION_ONLY
    res = oracle.localize(M, s, rg, score_frac=0.5, batch=batch, flags=flags | oracle.SEARCH_DFS)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), rg, flags)
    best, _ = oracle.brute_force(M, g, s)
    assert res.status == oracle.OK
    assert res.best_score == best
    assert M.score_nodes(g, s, [list(res.node)])[0] == best and res.node[6] == 0


@pytest.mark.parametrize("scan_index", [0, 2])
@pytest.mark.parametrize("batch", [1, 1000])
def test_dfs_exact_bound_roto_equals_brute_force(room, scan_index, batch):
    w, m, _, _ = room
    s, pose = synth.make_scan(1, scan_index)
    s = s[:200]
    rg = _window_ranges(pose)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), rg)
    e = g.exact_dilation(oracle.scan_dmax(s))
    M = oracle.Maps(m, w.r, w.levels, oracle.exact_flags(e))
    res = oracle.localize(M, s, rg, score_frac=0.3, batch=batch, flags=oracle.SEARCH_DFS)
    best, _ = oracle.brute_force(M, g, s)
    assert res.status == oracle.OK and res.best_score == best
    assert M.score_nodes(g, s, [list(res.node)])[0] == best and res.node[6] == 0


def test_dfs_and_best_first_differ_in_trajectory(room):
    """On the full room search (scan 1, b = 1000) the two orders expand
    different node sets in a different number of rounds; both return a leaf
    above the threshold, scored exactly."""
    w, m, _, _ = room
    s, _ = synth.make_scan(1, 1)
    M = oracle.Maps(m, w.r, w.levels)
    rg = oracle.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), rg)
    bfs = oracle.localize(M, s, rg, score_frac=w.score_frac, batch=1000)
    dfs = oracle.localize(M, s, rg, score_frac=w.score_frac, batch=1000, flags=oracle.SEARCH_DFS)
    assert bfs.status == dfs.status == oracle.OK
    assert (bfs.nodes_scored, bfs.iterations) != (dfs.nodes_scored, dfs.iterations)
    for r in (bfs, dfs):
        assert r.best_score >= math.ceil(w.score_frac * len(s))
        assert M.score_nodes(g, s, [list(r.node)])[0] == r.best_score and r.node[6] == 0


def test_dfs_full_room_reaches_threshold(room):
    """The depth-first order on the full room search (approximate rotational
    bound) still returns a leaf at or above the threshold, scored exactly."""
    w, m, s, pose = room
    M = oracle.Maps(m, w.r, w.levels)
    rg = oracle.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    res = oracle.localize(M, s, rg, score_frac=w.score_frac, batch=w.batch, flags=oracle.SEARCH_DFS)
    assert res.status == oracle.OK
    assert res.best_score >= math.ceil(w.score_frac * len(s))
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), rg)
    assert M.score_nodes(g, s, [list(res.node)])[0] == res.best_score and res.node[6] == 0


def test_dfs_threshold_not_reached(room):
    """No leaf reaches the threshold: NOT_FOUND, as for best-first."""
    w, m, s, _ = room
    M = oracle.Maps(m, w.r, w.levels)
    rg = oracle.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    far = s + 500.0   # d_max held at the room's scale: the far points widen no angle grid
    res = oracle.localize(M, far.astype(s.dtype), rg, score_frac=0.95, batch=w.batch, d_max=20.0,
                          flags=oracle.SEARCH_DFS)
    assert res.status == oracle.NOT_FOUND

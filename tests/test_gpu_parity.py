"""GPU (C-ABI) against the CPU oracle on the same seeded inputs.

Integer results are compared exactly: voxel-key sets per level, pose-grid
dimensions and rotation-table bits, Eq. (11) scores of arbitrary nodes and of
every child of branched parents, and the search's best score, match,
iteration count and number of nodes scored.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2310_10023_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_10023_gb300 import build, native
    build.build()
    native.load()
    return native


def _keyset(a):
    return set(map(tuple, np.asarray(a).reshape(-1, 3).tolist()))


def _sorted_keys(a):
    a = np.asarray(a, np.int64).reshape(-1, 3)
    return a[np.lexsort((a[:, 2], a[:, 1], a[:, 0]))]


@pytest.fixture(scope="module")
def room_pair(nv):
    w = synth.WORKLOADS["room"]
    m = synth.make_map(w.scene)
    return w, m, nv.bbs_build_maps(m, w.r, w.levels), oracle.Maps(m, w.r, w.levels)


def _ranges(nv, w, lo=None, hi=None, alo=None, ahi=None):
    lo, hi = lo or w.lo, hi or w.hi
    alo, ahi = alo or w.ang_lo, ahi or w.ang_hi
    return nv.make_ranges(lo, hi, alo, ahi), oracle.make_ranges(lo, hi, alo, ahi)


# ---- maps ------------------------------------------------------------------

def test_room_map_levels_equal_oracle(nv, room_pair):
    w, m, dm, om = room_pair
    for l in range(w.levels):   # every level's full key set
        assert np.array_equal(_sorted_keys(nv.bbs_maps_keys(dm, l)), _sorted_keys(om.keys(l))), l
        info = nv.bbs_maps_info(dm, l)
        assert info["voxels"] == om.count(l)
        assert info["buckets"] * 2 <= info["table_size"] * 1.0 + 1024


def test_undilated_leaf_and_device_input(nv):
    w = synth.WORKLOADS["room"]
    m = synth.make_map(w.scene)
    dm = nv.bbs_build_maps(torch.from_numpy(np.array(m)).cuda(), w.r, w.levels, nv.LEAF_UNDILATED)
    om = oracle.Maps(m, w.r, w.levels, oracle.LEAF_UNDILATED)
    for l in range(w.levels):
        assert _keyset(nv.bbs_maps_keys(dm, l)) == _keyset(om.keys(l)), l
    assert nv.bbs_maps_bbox(dm) == om.bbox()


@pytest.mark.parametrize("seed", [0, 1])
def test_random_cloud_maps_with_negative_keys(nv, seed):
    rng = np.random.default_rng(seed)
    pts = rng.normal(0, 30, size=(20000, 3)).astype(np.float32)
    pts[:50] = rng.uniform(-1e-3, 1e-3, size=(50, 3))          # around the zero boundary
    for r, L in ((0.37, 5), (2.0, 4)):
        dm = nv.bbs_build_maps(pts, r, L)
        om = oracle.Maps(pts, r, L)
        for l in range(L):
            assert _keyset(nv.bbs_maps_keys(dm, l)) == _keyset(om.keys(l)), (r, l)


def test_sparse_map_falls_back_to_hashed_levels(nv, room_pair):
    """The room map plus a copy 4.2 km away (3 km in x and y): the fine levels' boxes are then far
    too sparse for a byte grid, so the default layout hashes them (the
    coarsest levels may still qualify); key sets, scores and a search equal
    the oracle's."""
    w, m, _, _ = room_pair
    far = m + np.array([3000.0, 3000.0, 0.0], np.float32)
    both = np.concatenate([m, far]).astype(np.float32)
    dm = nv.bbs_build_maps(both, w.r, w.levels)
    om = oracle.Maps(both, w.r, w.levels)
    assert nv.bbs_maps_layout(dm, 0) in (nv.LAYOUT_COMPACT, nv.LAYOUT_WIDE)
    for l in range(w.levels):
        assert _keyset(nv.bbs_maps_keys(dm, l)) == _keyset(om.keys(l)), l
    s, _ = synth.make_scan(1, 0)
    nr, orr = _ranges(nv, w)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orr)
    nodes = _random_nodes(g, np.random.default_rng(8), 800, w.levels)
    assert np.array_equal(nv.bbs_score_batch(dm, s, nodes, nr), om.score_nodes(g, s, nodes))
    res = nv.bbs_localize(dm, s, nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch))
    _same_search(res, oracle.localize(om, s, orr, score_frac=w.score_frac, batch=w.batch))


def test_map_errors(nv):
    with pytest.raises(nv.BBSError) as e:
        nv.bbs_build_maps(np.array([[np.nan, 0, 0]], np.float32), 0.5, 2)
    assert e.value.code == nv.EINVAL
    with pytest.raises(nv.BBSError) as e:
        nv.bbs_build_maps(np.array([[3e6, 0, 0]], np.float32), 1.0, 2)
    assert e.value.code == nv.EKEYRANGE
    with pytest.raises(nv.BBSError):
        nv.bbs_build_maps(np.zeros((4, 3), np.float32), 0.5, 17)
    dm = nv.bbs_build_maps(np.zeros((0, 3), np.float32), 0.5, 2)
    assert nv.bbs_maps_info(dm, 0)["voxels"] == 0


# ---- pose grid -------------------------------------------------------------

@pytest.mark.parametrize("flags", [0, oracle.ANGLE_LOWER_EDGE, oracle.TRANSLATION_ONLY])
def test_pose_grid_bits_equal_oracle(nv, room_pair, flags):
    w, m, dm, om = room_pair
    s, _ = synth.make_scan(1, 0)
    nr, orr = _ranges(nv, w)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orr, flags)
    for l in range(w.levels):
        dims, A = nv.bbs_pose_grid(dm, s, nr, nv.make_opts(flags=flags), l)
        assert dims["N"] == g.N(l)
        assert dims["a"] == (g.a(l) if l > 0 else (1, 1, 1))
        assert (dims["wmin"], dims["wmax"]) == g.wrange()
        idx = np.arange(len(A)) if len(A) <= 4000 else np.random.default_rng(l).choice(len(A), 4000, replace=False)
        na, nb, ng = g.N(l)
        for t in idx:
            ia, ib, ig = t // (nb * ng), (t // ng) % nb, t % ng
            assert np.array_equal(A[t].view(np.uint32), g.rotation(l, ia, ib, ig).view(np.uint32)), (l, t)


@pytest.mark.parametrize("name", ["indoor", "outdoor"])
@pytest.mark.parametrize("flags", [0, oracle.ANGLE_LOWER_EDGE])
def test_search_rows_equal_oracle_bits(nv, name, flags):
    """The rows the search forms (FP32 double-float arithmetic, FP64 where it
    cannot decide the rounding; the pose grid's rows come from the same
    function) equal the oracle's FP64 rows bit for bit: every rotation of
    every level up to 60 k rotations, 60 k sampled beyond, on the indoor and
    outdoor grids, with segment-centre and lower-edge angles (the latter put
    exact zeros and rounding residues near 1e-17 into the tables)."""
    w = synth.WORKLOADS[name]
    s, _ = synth.make_scan(w.scene, 0)
    dm = nv.bbs_build_maps(np.array([[0.0, 0.0, 0.0], [5.0, 3.0, 1.0]], np.float32), w.r, w.levels)
    nr, orr = _ranges(nv, w)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orr, flags)
    for l in range(w.levels):
        dims, A = nv.bbs_pose_grid(dm, s, nr, nv.make_opts(flags=flags), l)
        assert dims["N"] == g.N(l)
        idx = np.arange(len(A)) if len(A) <= 60000 else np.random.default_rng(l).choice(len(A), 60000, replace=False)
        na, nb, ng = g.N(l)
        want = np.array([g.rotation(l, t // (nb * ng), (t // ng) % nb, t % ng) for t in idx])
        bad = np.nonzero((A[idx].view(np.uint32) != want.view(np.uint32)).any(axis=1))[0]
        assert len(bad) == 0, (l, idx[bad[:5]], A[idx[bad[:5]]], want[bad[:5]])


# ---- scores ----------------------------------------------------------------

def _random_nodes(g, rng, n, levels, tmin=-3, tmax=45):
    out = []
    for _ in range(n):
        l = int(rng.integers(0, levels))
        out.append([int(rng.integers(tmin >> l, (tmax >> l) + 1)), int(rng.integers(tmin >> l, (tmax >> l) + 1)),
                    int(rng.integers(-2, (12 >> l) + 1)), *(int(rng.integers(0, g.N(l)[i])) for i in range(3)), l])
    return np.array(out, np.int32)


@pytest.mark.parametrize("scan_index", [0, 3])
def test_score_batch_bit_exact_room(nv, room_pair, scan_index):
    w, m, dm, om = room_pair
    s, _ = synth.make_scan(1, scan_index)
    nr, orr = _ranges(nv, w)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orr)
    nodes = _random_nodes(g, np.random.default_rng(scan_index), 3000, w.levels)
    got = nv.bbs_score_batch(dm, s, nodes, nr)
    want = om.score_nodes(g, s, nodes)
    assert np.array_equal(got, want)
    # device-resident scan / nodes / scores
    gd = nv.bbs_score_batch(dm, torch.from_numpy(s).cuda(), torch.from_numpy(nodes).cuda(), nr)
    assert gd.is_cuda and np.array_equal(gd.cpu().numpy(), want)


def test_score_batch_ragged_and_edges(nv, room_pair):
    w, m, dm, om = room_pair
    s, _ = synth.make_scan(1, 1)
    nr, orr = _ranges(nv, w)
    for k in (1, 31, 33, 257, 999):
        sk = s[:k]
        g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(sk), orr)
        nodes = _random_nodes(g, np.random.default_rng(k), 200, w.levels, tmin=-(1 << 10), tmax=1 << 10)
        assert np.array_equal(nv.bbs_score_batch(dm, sk, nodes, nr), om.score_nodes(g, sk, nodes)), k
    # the extreme translations the grid allows: keys far outside the map miss
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orr)
    edge = np.array([[(1 << 20) >> l, -((1 << 20) >> l), 0, 0, 0, 0, l] for l in range(w.levels)], np.int32)
    assert np.array_equal(nv.bbs_score_batch(dm, s, edge, nr), om.score_nodes(g, s, edge))
    # empty node list
    assert len(nv.bbs_score_batch(dm, s, np.zeros((0, 7), np.int32), nr)) == 0


def test_score_batch_rejects_bad_nodes(nv, room_pair):
    w, m, dm, om = room_pair
    s, _ = synth.make_scan(1, 0)
    nr, _ = _ranges(nv, w)
    for bad in ([0, 0, 0, 0, 0, 0, 3], [0, 0, 0, -1, 0, 0, 0], [1 << 21, 0, 0, 0, 0, 0, 0]):
        with pytest.raises(nv.BBSError) as e:
            nv.bbs_score_batch(dm, s, np.array([bad], np.int32), nr)
        assert e.value.code == nv.EINVAL
    bad_scan = s.copy()
    bad_scan[5, 2] = np.nan
    with pytest.raises(nv.BBSError):
        nv.bbs_score_batch(dm, bad_scan, np.zeros((1, 7), np.int32), nr)
    # bbs_score_children: a size query (cap 0, no buffers) reports the count;
    # a sufficient cap with no output buffers is refused, not dereferenced
    import ctypes as C
    parents = np.array([[0, 0, 0, 0, 0, 0, w.levels - 1]], np.int32)
    sp = np.ascontiguousarray(s, np.float32)
    opts = nv.make_opts()
    cnt = C.c_int64(-1)
    lib = nv.load()
    args = (dm.h, C.c_void_p(sp.ctypes.data), len(sp), 0, C.byref(nr), C.byref(opts),
            C.c_void_p(parents.ctypes.data), 1)
    assert lib.bbs_score_children(*args, None, None, 0, C.byref(cnt)) == nv.EINVAL
    assert cnt.value > 0
    assert lib.bbs_score_children(*args, None, None, cnt.value, C.byref(cnt)) == nv.EINVAL
    assert b"NULL output" in lib.bbs_last_error()


@pytest.mark.parametrize("flags", [0, oracle.CHILD_LITERAL, oracle.TRANSLATION_ONLY])
def test_branch_kernel_children_bit_exact(nv, room_pair, flags):
    """The fused branch-and-score kernel: every child of every parent, in
    canonical order, with its Eq. (11) score."""
    w, m, dm, om = room_pair
    s, _ = synth.make_scan(1, 2)
    ang = ((-0.05, -0.05, 0.0), (0.05, 0.05, 2 * math.pi)) if flags & oracle.TRANSLATION_ONLY else (w.ang_lo, w.ang_hi)
    nr, orr = _ranges(nv, w, alo=ang[0], ahi=ang[1])
    opts = nv.make_opts(flags=flags)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orr, flags)
    rng = np.random.default_rng(flags)
    parents = _random_nodes(g, rng, 400, w.levels)
    parents[:, 6] = np.maximum(parents[:, 6], 1)
    for i, p in enumerate(parents):
        for a in range(3):
            parents[i, 3 + a] = min(p[3 + a], g.N(p[6])[a] - 1)
    nodes, scores = nv.bbs_score_children(dm, s, parents, nr, opts)
    want_nodes = np.concatenate([g.children(p) for p in parents])
    assert np.array_equal(nodes, want_nodes)
    assert np.array_equal(scores, om.score_nodes(g, s, want_nodes))


@pytest.mark.parametrize("layout", [0, 2])
def test_branch_kernel_chunk_edges(nv, layout):
    """The fused kernel stages the scan in 1568-point chunks, seven points per
    scoring thread (224 threads): scans that end on, just before and just
    after the chunk and thread-row boundaries (and the single point), under
    the byte-grid and the hashed layout, score every child as the oracle
    does."""
    w = synth.WORKLOADS["room"]
    m = synth.make_map(w.scene)
    om = oracle.Maps(m, w.r, w.levels)
    nv.bbs_set_probe_layout(layout)
    try:
        dm = nv.bbs_build_maps(m, w.r, w.levels)
    finally:
        nv.bbs_set_probe_layout(0)
    base, _ = synth.make_scan(1, 9, k=4200)
    nr, orr = _ranges(nv, w)
    for k in (1, 2, 3, 223, 224, 225, 448, 449, 1567, 1568, 1569, 1792, 3135, 3136, 3137, 4097):
        sk = np.ascontiguousarray(base[:k])
        g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(sk), orr)
        parents = _random_nodes(g, np.random.default_rng(k), 24, w.levels)
        parents[:, 6] = np.maximum(parents[:, 6], 1)
        for i, p in enumerate(parents):
            for a in range(3):
                parents[i, 3 + a] = min(p[3 + a], g.N(p[6])[a] - 1)
        nodes, scores = nv.bbs_score_children(dm, sk, parents, nr)
        assert np.array_equal(nodes, np.concatenate([g.children(p) for p in parents])), k
        assert np.array_equal(scores, om.score_nodes(g, sk, nodes)), (layout, k)


def test_branch_kernel_bit_exact_many_probes(nv, room_pair):
    """About a hundred million probes of the fused kernel against the oracle,
    element by element: 800 random parents over the room (levels 1 and 2,
    the whole rotation range), a 4200-point scan over three chunks.  A
    rotated coordinate rounded other than by the oracle's FP32 chain (for
    instance a product fused into the following sum) moves a floor across
    an integer about once in a few million probes, so a sample of this size
    catches it."""
    w, m, dm, om = room_pair
    s, _ = synth.make_scan(1, 9, k=4200)
    nr, orr = _ranges(nv, w)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orr)
    parents = _random_nodes(g, np.random.default_rng(77), 800, w.levels)
    parents[:, 6] = np.maximum(parents[:, 6], 1)
    for i, p in enumerate(parents):
        for a in range(3):
            parents[i, 3 + a] = min(p[3 + a], g.N(p[6])[a] - 1)
    nodes, scores = nv.bbs_score_children(dm, s, parents, nr)
    assert len(nodes) * len(s) > 5e7
    try:
        want = om.score_nodes(g, s, nodes, mt=True)
    except ImportError:   # no OpenMP build of the oracle
        want = om.score_nodes(g, s, nodes)
    bad = np.nonzero(scores != want)[0]
    assert len(bad) == 0, [(nodes[b].tolist(), int(scores[b]), int(want[b])) for b in bad[:5]]


# ---- search ----------------------------------------------------------------

def _same_search(res, ores):
    assert res.status == ores.status
    assert res.best_score == ores.best_score
    if ores.status == oracle.OK:
        assert list(res.node) == list(ores.node)
        assert np.allclose(list(res.pose), list(ores.pose), rtol=0, atol=1e-12)
    assert res.iterations == ores.iterations
    assert res.nodes_scored == ores.nodes_scored
    # Sec. IV-A's bound check along the same trajectory: the same children,
    # the same violations; the excess sums differ only in summation order
    assert res.children_scored == ores.children_scored
    assert res.bound_violations == ores.bound_violations
    assert math.isclose(res.bound_excess, ores.bound_excess, rel_tol=1e-9, abs_tol=1e-12)


@pytest.mark.parametrize("batch", [1, 500, 10000, 100000])
def test_room_localize_equals_oracle(nv, room_pair, batch):
    w, m, dm, om = room_pair
    s, pose = synth.make_scan(1, 0)
    nr, orr = _ranges(nv, w)
    if batch == 1:
        # sequential best-first on a window (the full room is slow for the oracle at b = 1)
        x0, y0 = math.floor(pose[0] / 2) * 2 - 2.0, math.floor(pose[1] / 2) * 2 - 2.0
        nr, orr = _ranges(nv, w, (x0, y0, 0.0), (x0 + 5.9, y0 + 5.9, 3.9),
                          (-0.05, -0.05, pose[5] - 0.2), (0.05, 0.05, pose[5] + 0.2))
    res = nv.bbs_localize(dm, s, nr, nv.make_opts(score_frac=w.score_frac, batch=batch))
    ores = oracle.localize(om, s, orr, score_frac=w.score_frac, batch=batch)
    _same_search(res, ores)
    assert res.status == nv.OK


@pytest.mark.parametrize("scan_index", [1, 2, 5])
def test_room_other_scans(nv, room_pair, scan_index):
    w, m, dm, om = room_pair
    s, pose = synth.make_scan(1, scan_index)
    nr, orr = _ranges(nv, w)
    res = nv.bbs_localize(dm, torch.from_numpy(s).cuda(), nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch))
    ores = oracle.localize(om, s, orr, score_frac=w.score_frac, batch=w.batch)
    _same_search(res, ores)


def test_translation_only_equals_brute_force(nv, room_pair):
    w, m, dm, om = room_pair
    s, pose = synth.make_scan(1, 1)
    s = s[:200]
    x0, y0 = math.floor(pose[0] / 2) * 2 - 2.0, math.floor(pose[1] / 2) * 2 - 2.0
    lo, hi = (x0, y0, 0.0), (x0 + 3.9, y0 + 3.9, 1.9)
    alo, ahi = (-0.02, -0.02, pose[5] - 0.12), (0.02, 0.02, pose[5] + 0.12)
    nr, orr = _ranges(nv, w, lo, hi, alo, ahi)
    flags = oracle.TRANSLATION_ONLY
    res = nv.bbs_localize(dm, s, nr, nv.make_opts(score_frac=0.5, batch=64, flags=flags))
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orr, flags)
    best, _ = oracle.brute_force(om, g, s)
    assert res.status == nv.OK and res.best_score == best
    ores = oracle.localize(om, s, orr, score_frac=0.5, batch=64, flags=flags)
    _same_search(res, ores)


def test_not_found_and_empty(nv, room_pair):
    w, m, dm, om = room_pair
    s, _ = synth.make_scan(1, 0)
    nr, orr = _ranges(nv, w)
    far = s.copy()
    far[:, 2] = np.float32(30.0)         # a plane 30 m above the room: no point can hit
    res = nv.bbs_localize(dm, far, nr, nv.make_opts(score_frac=0.5))
    assert res.status == nv.NOT_FOUND and res.found == 0
    res = nv.bbs_localize(dm, np.zeros((0, 3), np.float32), nr)
    assert res.status == nv.NOT_FOUND
    with pytest.raises(nv.BBSError):
        nv.bbs_localize(dm, s, nr, nv.make_opts(flags=nv.PRUNE_GE))


@pytest.mark.parametrize("levels", [1, 2])
def test_shallow_pyramids_equal_oracle(nv, levels):
    """Degenerate pyramids: with one level the initial set is the leaves
    themselves (the first pop ends the search), with two the search branches
    once; both follow the oracle exactly."""
    w = synth.WORKLOADS["room"]
    m = synth.make_map(w.scene)
    s, pose = synth.make_scan(w.scene, 0)
    s = np.ascontiguousarray(s[:300])
    x0, y0 = math.floor(pose[0] / 2) * 2 - 1.0, math.floor(pose[1] / 2) * 2 - 1.0
    lo, hi = (x0, y0, 0.0), (x0 + 3.9, y0 + 3.9, 2.9)
    alo, ahi = (-0.03, -0.03, pose[5] - 0.2), (0.03, 0.03, pose[5] + 0.2)
    dm = nv.bbs_build_maps(m, w.r, levels)
    om = oracle.Maps(m, w.r, levels)
    res = nv.bbs_localize(dm, s, nv.make_ranges(lo, hi, alo, ahi), nv.make_opts(score_frac=0.8, batch=2000))
    ores = oracle.localize(om, s, oracle.make_ranges(lo, hi, alo, ahi), score_frac=0.8, batch=2000)
    _same_search(res, ores)
    assert res.status == nv.OK


@pytest.mark.parametrize("kind", ["one_location", "origin_only"])
def test_degenerate_scans_equal_oracle(nv, room_pair, kind):
    """Scans whose points all sit at one location (every score is 0 or K)
    and a single point at the sensor origin (d_max = 0: one angle segment per
    axis at every level) follow the oracle exactly."""
    w, m, dm, om = room_pair
    s, pose = synth.make_scan(w.scene, 0)
    sc = np.repeat(s[5:6], 64, axis=0) if kind == "one_location" else np.zeros((1, 3), np.float32)
    x0, y0 = math.floor(pose[0] / 2) * 2 - 1.0, math.floor(pose[1] / 2) * 2 - 1.0
    lo, hi = (x0, y0, 0.0), (x0 + 3.9, y0 + 3.9, 2.9)
    alo, ahi = (-0.03, -0.03, pose[5] - 0.2), (0.03, 0.03, pose[5] + 0.2)
    res = nv.bbs_localize(dm, sc, nv.make_ranges(lo, hi, alo, ahi), nv.make_opts(score_frac=0.8, batch=2000))
    ores = oracle.localize(om, sc, oracle.make_ranges(lo, hi, alo, ahi), score_frac=0.8, batch=2000)
    _same_search(res, ores)
    assert res.status == nv.OK and res.best_score == len(sc)


def test_size_limits(nv, room_pair):
    """The largest inputs the ABI takes: a scan of more than 2^24 - 2 points
    (its score must fit the frontier key's 24-bit field) and more than 4096
    scans per bbs_localize_many call are refused before any device work, and
    the handle stays usable."""
    w, m, dm, om = room_pair
    nr, _ = _ranges(nv, w)
    big = torch.zeros(((1 << 24) - 1, 3), dtype=torch.float32, device="cuda")
    for fn in (nv.bbs_localize, nv.bbs_localize_hostqueue):
        with pytest.raises(nv.BBSError) as e:
            fn(dm, big, nr)
        assert e.value.code == nv.EINVAL and "2^24" in str(e.value), fn.__name__
    del big
    s, _ = synth.make_scan(1, 0)
    tiny = torch.from_numpy(s[:4]).cuda()
    with pytest.raises(nv.BBSError) as e:
        nv.bbs_localize_many(dm, [tiny] * 4097, nr)
    assert e.value.code == nv.EINVAL and "4096" in str(e.value)
    res = nv.bbs_localize(dm, s, nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch))
    assert res.status == nv.OK


def test_frontier_capacity_error(nv, room_pair):
    w, m, dm, om = room_pair
    s, _ = synth.make_scan(1, 0)
    nr, _ = _ranges(nv, w)
    with pytest.raises(nv.BBSError) as e:
        nv.bbs_localize(dm, s, nr, nv.make_opts(score_frac=0.3, batch=10 ** 7, max_frontier=1000))
    assert e.value.code == nv.ENOMEM
    # the handle stays usable after the error
    res = nv.bbs_localize(dm, s, nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch))
    assert res.status == nv.OK


# ---- batched searches ---------------------------------------------------------

def test_localize_many_equals_single(nv, room_pair):
    """Each scan of a batch gets exactly the result it gets alone."""
    w, m, dm, om = room_pair
    nr, _ = _ranges(nv, w)
    opts = nv.make_opts(score_frac=w.score_frac, batch=w.batch)
    scans = [synth.make_scan(1, i)[0] for i in range(6)]
    scans[2] = scans[2][:333]                       # uneven sizes
    scans[4] = synth.make_scan(1, 4, k=2500)[0]
    many = nv.bbs_localize_many(dm, [torch.from_numpy(s).cuda() for s in scans], nr, opts)
    for s, r in zip(scans, many):
        one = nv.bbs_localize(dm, s, nr, opts)
        assert (r.status, r.best_score, list(r.node), r.iterations, r.nodes_scored) == \
               (one.status, one.best_score, list(one.node), one.iterations, one.nodes_scored)


def test_localize_many_more_scans_than_slots(nv, room_pair):
    """300 scans: 256 advance together and the rest take the slots of
    searches that finish; every result is still the one it gets alone."""
    w, m, dm, om = room_pair
    nr, _ = _ranges(nv, w)
    opts = nv.make_opts(score_frac=w.score_frac, batch=w.batch)
    base = [synth.make_scan(1, i)[0] for i in range(12)]
    scans = [base[j % 12][: 200 + (37 * j) % 800] for j in range(300)]
    many = nv.bbs_localize_many(dm, scans, nr, opts)
    assert len(many) == 300
    for s, r in zip(scans, many):
        one = nv.bbs_localize(dm, s, nr, opts)
        assert (r.status, r.best_score, list(r.node), r.iterations, r.nodes_scored) == \
               (one.status, one.best_score, list(one.node), one.iterations, one.nodes_scored)


def test_localize_many_with_oracle(nv, room_pair):
    w, m, dm, om = room_pair
    nr, orr = _ranges(nv, w)
    scans = [synth.make_scan(1, i)[0] for i in (7, 8)]
    many = nv.bbs_localize_many(dm, scans, nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch))
    for s, r in zip(scans, many):
        _same_search(r, oracle.localize(om, s, orr, score_frac=w.score_frac, batch=w.batch))


def test_localize_many_uneven_indoor_scans_with_oracle(nv, indoor_pair):
    """The batched form on its own workload: 64 indoor scans of 2 k-30 k
    points (log-uniform, the benchmark's set) in one bbs_localize_many call.
    Four of them (the smallest, which the oracle finishes in seconds) against
    the CPU oracle's searches, run side by side on the host's cores; every
    result equals the scan localized alone on the GPU."""
    import oracle_pool
    w, m, dm, om = indoor_pair
    nr, orr = _ranges(nv, w)
    ks = synth.loguniform_sizes(4, 64, 2000, 30000)
    scans = [synth.make_scan(w.scene, 500 + i, k=int(k))[0] for i, k in enumerate(ks)]
    op = nv.make_opts(score_frac=w.score_frac, batch=w.batch)
    many = nv.bbs_localize_many(dm, [torch.from_numpy(s).cuda() for s in scans], nr, op)
    for s, r in zip(scans, many):
        a = nv.bbs_localize(dm, s, nr, op)
        assert (r.status, r.best_score, list(r.node), r.iterations, r.nodes_scored) == \
               (a.status, a.best_score, list(a.node), a.iterations, a.nodes_scored)
    pick = sorted(range(len(scans)), key=lambda i: len(scans[i]))[:4]
    jobs = [("indoor", scans[i], (w.lo, w.hi, w.ang_lo, w.ang_hi), w.score_frac, w.batch, 0, 0) for i in pick]
    for i, o in zip(pick, oracle_pool.localize_many(jobs)):
        r = many[i]
        assert (r.status, r.best_score, list(r.node), r.iterations, r.nodes_scored, r.children_scored,
                r.bound_violations) == (o["status"], o["best_score"], o["node"], o["iterations"], o["nodes_scored"],
                                        o["children_scored"], o["bound_violations"]), (i, len(scans[i]))


def test_frontier_grows_as_the_search_needs(nv, room_pair):
    """The frontier arrays start at 2^10 nodes and double when a round's
    survivors might not fit (the round waits while the host grows them):
    the searches are the ones run with the default capacity, in the graph loop,
    the host-driven loop and a multi-scan call; a cap below the search's need
    still fails with BBS_ENOMEM."""
    w, m, dm, om = room_pair
    nr, _ = _ranges(nv, w)
    scans = [synth.make_scan(w.scene, i)[0] for i in (0, 5)]

    def key(r):
        return (r.status, r.best_score, list(r.node), r.iterations, r.nodes_scored, r.peak_frontier,
                r.children_scored, r.bound_violations)

    op = nv.make_opts(score_frac=w.score_frac, batch=w.batch)
    base = [nv.bbs_localize(dm, s, nr, op) for s in scans]
    assert max(r.peak_frontier for r in base) > 4 << 10
    try:
        nv.bbs_set_tuning(frontier_log2=10)
        for flags in (0, nv.HOST_DRIVEN):
            o = nv.make_opts(score_frac=w.score_frac, batch=w.batch, flags=flags)
            for s, b in zip(scans, base):
                assert key(nv.bbs_localize(dm, s, nr, o)) == key(b), flags
        many = nv.bbs_localize_many(dm, scans, nr, op)
        for r, b in zip(many, base):
            assert (r.status, r.best_score, list(r.node), r.iterations, r.nodes_scored) == \
                   (b.status, b.best_score, list(b.node), b.iterations, b.nodes_scored)
        with pytest.raises(nv.BBSError) as e:
            nv.bbs_localize(dm, scans[0], nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch,
                                                           max_frontier=2048))
        assert e.value.code == nv.ENOMEM
    finally:
        nv.bbs_set_tuning(reset=True)


def test_launch_log_matches_the_timed_result(nv, room_pair):
    """bbs_launch_log lists the timed call's scoring launches: as many as the
    result reports, their units summing to its gathers (tasks x scan points)
    and their milliseconds to its scoring time."""
    w, m, dm, om = room_pair
    nr, _ = _ranges(nv, w)
    s, _ = synth.make_scan(w.scene, 1)
    r = nv.bbs_localize(dm, s, nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch, flags=nv.TIME_KERNELS))
    units, ms = nv.bbs_launch_log()
    assert len(units) == r.score_launches > 1
    assert int(units.sum()) == r.gathers
    assert math.isclose(float(ms.sum()), r.score_ms, rel_tol=1e-5)
    assert (units > 0).all() and (ms > 0).all()


def test_localize_many_empty_and_not_found(nv, room_pair):
    w, m, dm, om = room_pair
    nr, _ = _ranges(nv, w)
    s, _ = synth.make_scan(1, 0)
    far = s.copy()
    far[:, 2] = np.float32(30.0)
    res = nv.bbs_localize_many(dm, [s, np.zeros((0, 3), np.float32), far], nr,
                               nv.make_opts(score_frac=0.6, batch=w.batch))
    assert res[0].status == nv.OK
    assert res[1].status == nv.NOT_FOUND
    assert res[2].status == nv.NOT_FOUND


# ---- every bucket layout --------------------------------------------------------

@pytest.mark.parametrize("layout", [0, 1, 2, 3, 4])
def test_layouts_agree_with_oracle(nv, layout):
    w = synth.WORKLOADS["room"]
    m = synth.make_map(w.scene)
    om = oracle.Maps(m, w.r, w.levels)
    nv.bbs_set_probe_layout(layout)
    try:
        dm = nv.bbs_build_maps(m, w.r, w.levels)
    finally:
        nv.bbs_set_probe_layout(0)
    # the room's boxes are small: every layout applies
    want = {0: nv.LAYOUT_BYTES, 1: nv.LAYOUT_WIDE, 2: nv.LAYOUT_COMPACT, 3: nv.LAYOUT_DENSE, 4: nv.LAYOUT_BYTES}[layout]
    assert [nv.bbs_maps_layout(dm, l) for l in range(w.levels)] == [want] * w.levels
    for l in range(w.levels):
        assert _keyset(nv.bbs_maps_keys(dm, l)) == _keyset(om.keys(l)), (layout, l)
    s, _ = synth.make_scan(1, 6)
    nr, orr = _ranges(nv, w)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orr)
    nodes = _random_nodes(g, np.random.default_rng(40 + layout), 1500, w.levels)
    assert np.array_equal(nv.bbs_score_batch(dm, s, nodes, nr), om.score_nodes(g, s, nodes))
    parents = nodes[nodes[:, 6] > 0][:200]
    kn, ks = nv.bbs_score_children(dm, s, parents, nr)
    assert np.array_equal(ks, om.score_nodes(g, s, kn))
    res = nv.bbs_localize(dm, s, nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch))
    _same_search(res, oracle.localize(om, s, orr, score_frac=w.score_frac, batch=w.batch))


# ---- full-size workloads ----------------------------------------------------------

@pytest.fixture(scope="module")
def indoor_pair(nv):
    w = synth.WORKLOADS["indoor"]
    m = synth.make_map(w.scene)
    return w, m, nv.bbs_build_maps(torch.from_numpy(np.array(m)).cuda(), w.r, w.levels), oracle.Maps(m, w.r, w.levels)


def test_indoor_maps_and_scores_bit_exact(nv, indoor_pair):
    w, m, dm, om = indoor_pair
    for l in range(w.levels):
        assert nv.bbs_maps_info(dm, l)["voxels"] == om.count(l)
    for l in range(w.levels):
        assert _keyset(nv.bbs_maps_keys(dm, l)) == _keyset(om.keys(l)), l
    s, _ = synth.make_scan(2, 0)
    nr, orr = _ranges(nv, w)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orr)
    nodes = _random_nodes(g, np.random.default_rng(9), 600, w.levels, tmin=-5, tmax=500)
    assert np.array_equal(nv.bbs_score_batch(dm, s, nodes, nr), om.score_nodes(g, s, nodes))
    parents = nodes[nodes[:, 6] > 0][:60]
    kn, ks = nv.bbs_score_children(dm, torch.from_numpy(s).numpy(), parents, nr)
    assert np.array_equal(ks, om.score_nodes(g, s, kn))


def test_indoor_localize_equals_oracle(nv, indoor_pair):
    """A full-size indoor search (8 k points, 6 levels, b = 16384): the GPU
    follows the oracle's trajectory exactly."""
    w, m, dm, om = indoor_pair
    s, pose = synth.make_scan(2, 1)
    nr, orr = _ranges(nv, w)
    res = nv.bbs_localize(dm, torch.from_numpy(s).cuda(), nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch))
    ores = oracle.localize(om, s, orr, score_frac=w.score_frac, batch=w.batch)
    _same_search(res, ores)
    assert res.status == nv.OK
    from planted import check_planted
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orr)
    steps = check_planted(w.r, g, om, s, pose, list(res.node), res.best_score, list(res.pose))
    assert max(steps) <= 1.0   # this scan resolves every angle to one step


@pytest.fixture(scope="module")
def outdoor_pair(nv):
    w = synth.WORKLOADS["outdoor"]
    m = synth.make_map(w.scene)
    return w, m, nv.bbs_build_maps(torch.from_numpy(np.array(m)).cuda(), w.r, w.levels), oracle.Maps(m, w.r, w.levels)


def test_exact_bound_indoor_window_equals_oracle(nv):
    """The exact-bound mode on indoor data: the indoor map cropped to 32 x 32 m
    around the planted pose of scan 1, the scan's points within 10 m (every
    4th), a window of level-5 cells (6.4 m) around the pose, roll / pitch
    +-0.02 rad and yaw +-0.05 rad.  Maps widened by the required e; the GPU
    search (whose frontier grows past its start) follows the oracle's exactly."""
    w = synth.WORKLOADS["indoor"]
    m = synth.make_map(w.scene)
    s, pose = synth.make_scan(w.scene, 1)
    R5 = w.r * 32
    kx, ky = math.floor(pose[0] / R5), math.floor(pose[1] / R5)
    cx, cy = (kx + 0.5) * R5, (ky + 0.5) * R5
    crop = np.ascontiguousarray(m[(np.abs(m[:, 0] - cx) < 16) & (np.abs(m[:, 1] - cy) < 16)])
    near = np.ascontiguousarray(s[np.linalg.norm(s, axis=1) < 10.0][::4])
    lo, hi = (kx * R5, ky * R5, 0.0), (kx * R5, ky * R5, 0.0)
    alo, ahi = (-0.02, -0.02, pose[5] - 0.05), (0.02, 0.02, pose[5] + 0.05)
    nr, orr = nv.make_ranges(lo, hi, alo, ahi), oracle.make_ranges(lo, hi, alo, ahi)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(near), orr)
    e = g.exact_dilation(oracle.scan_dmax(near))
    dme = nv.bbs_build_maps(crop, w.r, w.levels, nv.exact_bound_flags(e))
    assert nv.bbs_exact_dilation(dme, near, nr, nv.make_opts()) == e
    ome = oracle.Maps(crop, w.r, w.levels, oracle.exact_flags(e))
    for l in range(w.levels):
        assert np.array_equal(_sorted_keys(nv.bbs_maps_keys(dme, l)), _sorted_keys(ome.keys(l))), l
    try:
        nv.bbs_set_tuning(frontier_log2=12)
        res = nv.bbs_localize(dme, near, nr, nv.make_opts(score_frac=0.8, batch=w.batch))
    finally:
        nv.bbs_set_tuning(reset=True)
    ores = oracle.localize(ome, near, orr, score_frac=0.8, batch=w.batch)
    _same_search(res, ores)
    assert res.status == nv.OK and res.peak_frontier > 1 << 12


def test_outdoor_search_equals_oracle(nv, outdoor_pair):
    """The outdoor workload's own search (800 x 800 x 40 m city, 40 M map
    points, r = 1 m, 8 levels, the 400 x 400 x 10 m window, full yaw) with
    the scan thinned to every 10th of its 20 k points (the oracle's search of
    the whole scan takes minutes on one core): the GPU follows the oracle's
    trajectory exactly -- best score, match, iterations, nodes scored and the
    bound check."""
    w, m, dm, om = outdoor_pair
    s, pose = synth.make_scan(3, 2)
    s = np.ascontiguousarray(s[::10])
    nr, orr = _ranges(nv, w)
    res = nv.bbs_localize(dm, torch.from_numpy(s).cuda(), nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch))
    ores = oracle.localize(om, s, orr, score_frac=w.score_frac, batch=w.batch)
    _same_search(res, ores)
    assert res.status == nv.OK and res.best_score >= math.ceil(w.score_frac * len(s))


def test_outdoor_sampled_parity_and_planted_pose(nv, outdoor_pair):
    """800 x 800 x 40 m city, 40 M map points, 20 k-point scan: sampled scores
    bit-exact, the returned leaf's oracle score equals the reported best, and
    the planted pose is recovered."""
    w, m, dm, om = outdoor_pair
    s, pose = synth.make_scan(3, 2)
    nr, orr = _ranges(nv, w)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orr)
    nodes = _random_nodes(g, np.random.default_rng(3), 200, w.levels, tmin=150, tmax=650)
    assert np.array_equal(nv.bbs_score_batch(dm, s, nodes, nr), om.score_nodes(g, s, nodes))
    res = nv.bbs_localize(dm, torch.from_numpy(s).cuda(), nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch))
    assert res.status == nv.OK
    assert om.score_nodes(g, s, [list(res.node)])[0] == res.best_score
    from planted import check_planted
    check_planted(w.r, g, om, s, pose, list(res.node), res.best_score, list(res.pose))


# ---- the device-driven iteration loop --------------------------------------------

def test_graph_loop_equals_host_loop(nv, room_pair, indoor_pair):
    """The captured-graph loop (default) and the host-driven loop follow the
    same trajectory: identical results, iterations and nodes scored."""
    for (w, m, dm, om), idx in ((room_pair, 3), (indoor_pair, 4)):
        s, _ = synth.make_scan(w.scene, idx)
        nr, _ = _ranges(nv, w)
        a = nv.bbs_localize(dm, s, nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch))
        b = nv.bbs_localize(dm, s, nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch, flags=nv.HOST_DRIVEN))
        assert (a.status, a.best_score, list(a.node), a.iterations, a.nodes_scored, a.peak_frontier) == \
               (b.status, b.best_score, list(b.node), b.iterations, b.nodes_scored, b.peak_frontier)
    w, m, dm, om = indoor_pair
    nr, _ = _ranges(nv, w)
    scans = [synth.make_scan(2, 70 + i, k=3000 + 2500 * i)[0] for i in range(5)]
    many = nv.bbs_localize_many(dm, scans, nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch))
    many_h = nv.bbs_localize_many(dm, scans, nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch,
                                                              flags=nv.HOST_DRIVEN))
    for a, b in zip(many, many_h):
        assert (a.status, a.best_score, list(a.node), a.iterations, a.nodes_scored) == \
               (b.status, b.best_score, list(b.node), b.iterations, b.nodes_scored)


def test_launch_shape_does_not_change_results(nv, room_pair, indoor_pair):
    """Rounds split into many small launches (the host-planned windows of a
    round above the launch capacity), other static shares, grab sizes and CTA
    counts: every result, iteration count and node count is unchanged, on the
    graph loop and the host loop, for one search and for several at once."""
    def key(r):
        return (r.status, r.best_score, list(r.node), r.iterations, r.nodes_scored, r.peak_frontier)

    w, m, dm, om = indoor_pair
    nr, _ = _ranges(nv, w)
    scans = [synth.make_scan(2, 90 + i, k=2500 + 2000 * i)[0] for i in range(3)]
    rw, rm, rdm, rom = room_pair
    rnr, _ = _ranges(nv, rw)
    rscan = synth.make_scan(rw.scene, 5)[0]
    opts = nv.make_opts(score_frac=w.score_frac, batch=w.batch)
    ropts = nv.make_opts(score_frac=rw.score_frac, batch=rw.batch)
    base = [key(nv.bbs_localize(dm, s, nr, opts)) for s in scans] + [key(nv.bbs_localize(rdm, rscan, rnr, ropts))]
    base_many = [key(r) for r in nv.bbs_localize_many(dm, scans, nr, opts)]
    try:
        for shape in ({"launch_tasks": 64}, {"launch_tasks": 1000, "static_pm": 1, "grab_min": 1},
                      {"static_pm": 1000, "ctas_per_sm": 1}, {"launch_tasks": 333, "grab_min": 4096, "ctas_per_sm": 3}):
            nv.bbs_set_tuning(**shape)
            got = nv.bbs_get_tuning()
            for k, v in shape.items():
                assert got[k] == v
            for flags in (0, nv.HOST_DRIVEN):
                o = nv.make_opts(score_frac=w.score_frac, batch=w.batch, flags=flags)
                ro = nv.make_opts(score_frac=rw.score_frac, batch=rw.batch, flags=flags)
                res = [key(nv.bbs_localize(dm, s, nr, o)) for s in scans] + [key(nv.bbs_localize(rdm, rscan, rnr, ro))]
                assert res == base, (shape, flags)
                assert [key(r) for r in nv.bbs_localize_many(dm, scans, nr, o)] == base_many, (shape, flags)
    finally:
        nv.bbs_set_tuning(reset=True)
    assert nv.bbs_get_tuning() == {"launch_tasks": 1 << 19, "static_pm": 750, "grab_min": 16, "ctas_per_sm": 4,
                                   "frontier_log2": 0}


# ---- exact-bound mode --------------------------------------------------------

def _window(pose, half_yaw=0.12, rp=0.02):
    x0 = math.floor(pose[0] / 2.0) * 2.0 - 2.0
    y0 = math.floor(pose[1] / 2.0) * 2.0 - 2.0
    return (x0, y0, 0.0), (x0 + 3.9, y0 + 3.9, 1.9), (-rp, -rp, pose[5] - half_yaw), (rp, rp, pose[5] + half_yaw)


@pytest.mark.parametrize("leaf", [0, oracle.LEAF_UNDILATED])
def test_exact_bound_maps_and_search_equal_oracle(nv, leaf):
    """Exact-bound maps: every level's key set equals the oracle's (levels above
    the leaves widened by e); the requirement the library reports equals the
    oracle's; localize on a window equals the oracle's exact BnB (which the
    oracle pins equal to the exhaustive maximum); a map widened too little is
    refused."""
    w = synth.WORKLOADS["room"]
    m = synth.make_map(w.scene)
    s, pose = synth.make_scan(1, 0)
    s = s[:200]
    lo, hi, alo, ahi = _window(pose)
    nr, orr = nv.make_ranges(lo, hi, alo, ahi), oracle.make_ranges(lo, hi, alo, ahi)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orr, leaf)
    e = g.exact_dilation(oracle.scan_dmax(s))
    dm = nv.bbs_build_maps(m, w.r, w.levels, leaf | nv.exact_bound_flags(e))
    om = oracle.Maps(m, w.r, w.levels, leaf | oracle.exact_flags(e))
    for l in range(w.levels):
        assert _keyset(nv.bbs_maps_keys(dm, l)) == _keyset(om.keys(l)), l
    assert nv.bbs_exact_dilation(dm, s, nr, nv.make_opts(flags=leaf)) == e
    for batch in (1, 1000):
        r = nv.bbs_localize(dm, s, nr, nv.make_opts(score_frac=0.3, batch=batch, flags=leaf))
        o = oracle.localize(om, s, orr, score_frac=0.3, batch=batch, flags=leaf)
        assert (r.status, r.best_score, list(r.node), r.iterations, r.nodes_scored) == \
               (o.status, o.best_score, list(o.node), o.iterations, o.nodes_scored), batch
    small = nv.bbs_build_maps(m, w.r, w.levels, leaf | nv.exact_bound_flags(e - 1))
    with pytest.raises(nv.BBSError) as ex:
        nv.bbs_localize(small, s, nr, nv.make_opts(score_frac=0.3, flags=leaf))
    assert ex.value.code == nv.EINVAL
    with pytest.raises(nv.BBSError) as ex:
        nv.bbs_localize(dm, s, nr, nv.make_opts(score_frac=0.3, flags=leaf | nv.CHILD_LITERAL))
    assert ex.value.code == nv.EINVAL


# ---- the frontier on the host (Algorithm 2's own layout) -----------------------

def test_host_queue_equals_device_frontier(nv, room_pair, indoor_pair):
    """The host-queue search (per-batch copies, host buckets) follows the same
    canonical iteration as the CPU oracle (room scans) and the device-resident
    engine: identical results and counts, also when rounds are split into
    small launches."""
    def key(r):
        return (r.status, r.best_score, list(r.node), r.iterations, r.nodes_scored, r.peak_frontier,
                r.children_scored, r.bound_violations)

    cases = []
    w, m, dm, om = room_pair
    nr, orr = _ranges(nv, w)
    for i in (0, 3):
        s = synth.make_scan(w.scene, i)[0]
        cases.append((dm, s, nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch)))
        ores = oracle.localize(om, s, orr, score_frac=w.score_frac, batch=w.batch)
        res = nv.bbs_localize_hostqueue(dm, s, nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch))
        _same_search(res, ores)
        assert res.peak_frontier == ores.peak_frontier
    w, m, dm, om = indoor_pair
    nr, _ = _ranges(nv, w)
    cases.append((dm, synth.make_scan(w.scene, 2)[0], nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch)))
    for maps, s, rg, op in cases:
        a = nv.bbs_localize(maps, s, rg, op)
        b = nv.bbs_localize_hostqueue(maps, s, rg, op)
        assert key(a) == key(b)
        assert b.h2d_bytes > a.h2d_bytes and b.d2h_bytes > a.d2h_bytes   # the per-batch copies
    try:
        nv.bbs_set_tuning(launch_tasks=100)
        maps, s, rg, op = cases[0]
        assert key(nv.bbs_localize_hostqueue(maps, s, rg, op)) == key(nv.bbs_localize(maps, s, rg, op))
    finally:
        nv.bbs_set_tuning(reset=True)


# ---- depth-first order (Table I's DFS), host queue ------------------------------

def _dfs_cases(nv, room_pair):
    w, m, dm, om = room_pair
    nr, orr = _ranges(nv, w)
    cases = [("room scan 1, b 1000", dm, om, synth.make_scan(1, 1)[0], nr, orr, w.score_frac, 1000, 0),
             ("room scan 0, b 10000", dm, om, synth.make_scan(1, 0)[0], nr, orr, w.score_frac, w.batch, 0)]
    s, pose = synth.make_scan(1, 2)
    s = s[:200]
    lo, hi, alo, ahi = _window(pose)
    wnr, worr = _ranges(nv, w, lo, hi, alo, ahi)
    for b in (1, 64):
        cases.append((f"window, translation only, b {b}", dm, om, s, wnr, worr, 0.5, b, oracle.TRANSLATION_ONLY))
    return cases


@pytest.mark.parametrize("idx", [0, 1, 2, 3])
def test_dfs_host_queue_equals_oracle(nv, room_pair, idx):
    """The depth-first order of the host-queue search reproduces the oracle's:
    same match, best, rounds, nodes scored and peak frontier."""
    name, dm, om, s, nr, orr, frac, batch, flags = _dfs_cases(nv, room_pair)[idx]
    res = nv.bbs_localize_hostqueue(dm, s, nr, nv.make_opts(score_frac=frac, batch=batch, flags=flags | nv.SEARCH_DFS))
    ores = oracle.localize(om, s, orr, score_frac=frac, batch=batch, flags=flags | oracle.SEARCH_DFS)
    _same_search(res, ores)
    assert res.peak_frontier == ores.peak_frontier, name
    assert res.status == nv.OK


def test_dfs_exact_bound_equals_brute_force_on_gpu(nv, room_pair):
    """Exact-bound maps: the depth-first order on the GPU returns the
    exhaustive optimum, as the oracle's does, and equals the oracle's run."""
    w, m, dm, om = room_pair
    s, pose = synth.make_scan(1, 0)
    s = s[:200]
    lo, hi, alo, ahi = _window(pose)
    nr, orr = _ranges(nv, w, lo, hi, alo, ahi)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orr)
    e = g.exact_dilation(oracle.scan_dmax(s))
    dme = nv.bbs_build_maps(m, w.r, w.levels, nv.exact_bound_flags(e))
    ome = oracle.Maps(m, w.r, w.levels, oracle.exact_flags(e))
    res = nv.bbs_localize_hostqueue(dme, s, nr, nv.make_opts(score_frac=0.3, batch=100, flags=nv.SEARCH_DFS))
    ores = oracle.localize(ome, s, orr, score_frac=0.3, batch=100, flags=oracle.SEARCH_DFS)
    best, _ = oracle.brute_force(ome, g, s)
    _same_search(res, ores)
    assert res.best_score == best


def test_dfs_refused_by_device_engine(nv, room_pair):
    w, m, dm, om = room_pair
    s, _ = synth.make_scan(1, 0)
    nr, _ = _ranges(nv, w)
    with pytest.raises(nv.BBSError) as e:
        nv.bbs_localize(dm, s, nr, nv.make_opts(score_frac=w.score_frac, batch=w.batch, flags=nv.SEARCH_DFS))
    assert e.value.code == nv.EINVAL


def test_engine_switches_kernel_variant_with_the_maps(nv, room_pair):
    """Byte-grid maps and hashed maps used alternately by the cached engines:
    the loop graph is recaptured with the matching scoring kernel each time,
    and every result equals the oracle's."""
    w, m, dm, om = room_pair
    nv.bbs_set_probe_layout(2)
    try:
        hashed = nv.bbs_build_maps(m, w.r, w.levels)
    finally:
        nv.bbs_set_probe_layout(0)
    assert nv.bbs_maps_layout(hashed, 0) == nv.LAYOUT_COMPACT and nv.bbs_maps_layout(dm, 0) == nv.LAYOUT_BYTES
    nr, orr = _ranges(nv, w)
    op = nv.make_opts(score_frac=w.score_frac, batch=w.batch)
    for i, maps in enumerate([dm, hashed, dm, hashed]):
        s, _ = synth.make_scan(1, i % 2)
        ores = oracle.localize(om, s, orr, score_frac=w.score_frac, batch=w.batch)
        _same_search(nv.bbs_localize(maps, s, nr, op), ores)

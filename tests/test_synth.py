"""The seeded input generator: reproducible random stream and workload shapes."""
import json
import math
import os

import numpy as np

from paper_2310_10023_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_mt19937_64_published_value():
    g = json.load(open(os.path.join(GOLD, "mt19937_64.json")))
    out = synth.mt64(g["seed"], g["index"])
    assert int(out[-1]) == g["value"]


def test_room_map_and_scan_shapes():
    m = synth.make_map(1)
    assert 3.0e5 < len(m) < 4.5e5
    assert np.all(m.min(0) >= -1e-6) and np.all(m.max(0) <= np.array([20, 20, 5]) + 1e-6)
    s, pose = synth.make_scan(1, 0)
    assert s.shape == (1000, 3) and s.dtype == np.float32
    assert 0.5 <= pose[0] <= 19.5 and 0.5 <= pose[1] <= 19.5 and pose[2] == 1.0
    assert abs(pose[3]) <= 2 * math.pi / 180 and abs(pose[4]) <= 2 * math.pi / 180
    assert np.isfinite(s).all()


def test_deterministic():
    a, pa = synth.make_scan(1, 3)
    b, pb = synth.make_scan(1, 3)
    assert np.array_equal(a, b) and pa == pb
    c, _ = synth.make_scan(1, 4)
    assert not np.array_equal(a, c)


def test_exact_size_scans():
    for k in (2000, 5123):
        s, _ = synth.make_scan(1, 0, k=k)
        assert s.shape == (k, 3)


def test_scan_points_lie_on_map_surfaces():
    # transform the scan by its planted pose; noise-free it would sit on the
    # sampled surfaces, so most points must lie within 10 cm of a map point
    from scipy.spatial import cKDTree
    from scipy.spatial.transform import Rotation
    m = synth.make_map(1)
    s, pose = synth.make_scan(1, 2)
    R = Rotation.from_euler("ZYX", [pose[5], pose[4], pose[3]]).as_matrix()
    w = s.astype(np.float64) @ R.T + np.array(pose[:3])
    d, _ = cKDTree(m).query(w)
    assert np.mean(d < 0.1) > 0.9


def test_trace_is_poisson_and_loguniform():
    arr, ks = synth.poisson_trace(7, 50.0, 4000)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert abs(gaps.mean() - 1 / 50.0) < 0.002
    assert ks.min() >= 2000 and ks.max() <= 30000
    lk = np.log(ks)
    assert abs(lk.mean() - (math.log(2000) + math.log(30000)) / 2) < 0.05

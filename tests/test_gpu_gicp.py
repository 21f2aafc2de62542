"""GICP refinement on the GPU (bbs_gicp, bbs_gicp_linearize) against the
oracle (oracle/gicp.py): correspondences bit-exact, linearizations within
FP64 summation-order tolerance, whole runs to the same pose."""
import math

import numpy as np
import pytest

import oracle
from oracle import gicp
from paper_2310_10023_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_10023_gb300 import native
    native.load()
    return native


@pytest.fixture(scope="module")
def room(nv):
    w = synth.WORKLOADS["room"]
    m = synth.make_map(1)
    dt = nv.bbs_gicp_target_build(m, w.r)
    ot = gicp.Target(m, w.r)
    return ot.r, dt, ot.keys, ot


def test_target_equals_oracle(nv, room):
    r, dt, keys, ot = room
    info = nv.bbs_gicp_target_info(dt)
    assert info["voxels"] == len(ot.keys)
    assert info["table_size"] >= 2 * info["voxels"] // 2 and info["max_probe"] < 64


def _start(pose, dt=(0.1, -0.07, 0.04), dw=(0.01, -0.008, 0.02)):
    R, t = gicp.pose_to_rt(pose)
    return gicp.exp_so3(np.array(dw)) @ R, t + np.array(dt)


@pytest.mark.parametrize("scan_index", [0, 1, 2])
@pytest.mark.parametrize("offset", [0, 1])
def test_linearization_equals_oracle(nv, room, scan_index, offset):
    r, dt, keys, occ = room
    s, pose = synth.make_scan(1, scan_index)
    s64 = s.astype(np.float64)
    R, t = _start(pose) if offset else gicp.pose_to_rt(pose)
    H, g, cost, n, vox, found = nv.bbs_gicp_linearize(dt, s, R, t)
    Cs = gicp.source_covariances(s64, 2 * r, r, 1e-3)
    lin = gicp.linearize(occ, s64, Cs, R, t, r, r, 1e-3)
    assert np.array_equal(found, lin.found)
    assert np.array_equal(vox[found], lin.voxels[lin.found])
    assert n == lin.n and n > len(s) // 2
    assert np.allclose(H, lin.H, rtol=1e-10, atol=1e-9 * np.abs(lin.H).max())
    assert np.allclose(g, lin.g, rtol=1e-10, atol=1e-9 * np.abs(lin.g).max())
    assert math.isclose(cost, lin.cost, rel_tol=1e-10)


@pytest.mark.parametrize("scan_index", [0, 3])
def test_run_equals_oracle(nv, room, scan_index):
    r, dt, keys, occ = room
    s, pose = synth.make_scan(1, scan_index)
    R0, t0 = _start(pose)
    res = nv.bbs_gicp(dt, s, R0, t0)
    o = gicp.gicp(occ, s.astype(np.float64), R0, t0, r)
    assert res.status == nv.OK
    assert (res.iterations, bool(res.converged), res.correspondences) == (o.iterations, o.converged, o.n)
    Rg, tg = res.Rt()
    assert np.allclose(Rg, o.R, atol=1e-9) and np.allclose(tg, o.t, atol=1e-8)
    assert math.isclose(res.cost, o.cost, rel_tol=1e-8)
    assert np.allclose(res.pose, gicp.rt_to_pose(o.R, o.t), atol=1e-8)


def test_recovers_planted_pose(nv, room):
    """Voxel centres seen from a known pose: recovered from 0.12 m / 0.03 rad off."""
    r, dt, keys, occ = room
    rng = np.random.default_rng(4)
    R = gicp.rot_zyx(0.01, -0.015, 2.1)
    t = np.array([9.0, 8.5, 1.2])
    sel = occ.centroid[rng.choice(len(keys), 800, replace=False)]
    s = ((sel - t) @ R).astype(np.float32)
    R0 = gicp.exp_so3(np.array([0.01, -0.01, 0.025])) @ R
    res = nv.bbs_gicp(dt, s, R0, t + np.array([0.12, -0.08, 0.05]), nv.make_gicp_opts(max_iters=40))
    Rg, tg = res.Rt()
    assert res.converged and np.linalg.norm(tg - t) < 1e-4 and np.linalg.norm(Rg - R) < 1e-5


def test_device_input_and_errors(nv, room):
    torch = pytest.importorskip("torch")
    r, dt, keys, occ = room
    s, pose = synth.make_scan(1, 1)
    R0, t0 = _start(pose)
    a = nv.bbs_gicp(dt, s, R0, t0)
    b = nv.bbs_gicp(dt, torch.from_numpy(s).cuda(), R0, t0)
    assert np.array_equal(np.array(a.R), np.array(b.R)) and np.array_equal(np.array(a.t), np.array(b.t))
    with pytest.raises(nv.BBSError) as e:
        nv.bbs_gicp(dt, np.zeros((0, 3), np.float32), R0, t0)
    assert e.value.code == nv.EINVAL
    bad = synth.make_map(1)[:100].copy()
    bad[5, 0] = np.nan
    with pytest.raises(nv.BBSError) as e:
        nv.bbs_gicp_target_build(bad, 0.5)
    assert e.value.code == nv.EKEYRANGE


def test_refines_the_bnb_estimate_indoor(nv):
    """Indoor: the BnB leaf (a voxel-resolution pose) refined by GICP lies
    closer to the planted pose on every scan, to within a few centimetres
    (the map's surface samples are averaged per 0.2 m voxel; the scans carry
    3 cm noise)."""
    w = synth.WORKLOADS["indoor"]
    m = synth.make_map(w.scene)
    dm = nv.bbs_build_maps(m, w.r, w.levels)
    d0 = nv.bbs_gicp_target_build(m, w.r)
    a = nv.workload_args(w)
    better = 0
    errs = []
    for i in range(3):
        s, pose = synth.make_scan(w.scene, i)
        res = nv.bbs_localize(dm, s, a.ranges, a.opts)
        assert res.status == nv.OK
        R0, t0 = gicp.pose_to_rt(list(res.pose))
        g = nv.bbs_gicp(d0, s, R0, t0, nv.make_gicp_opts(max_iters=30))
        assert g.status == nv.OK and g.correspondences > len(s) // 2
        e0 = np.linalg.norm(t0 - np.array(pose[:3]))
        e1 = np.linalg.norm(np.array(g.t) - np.array(pose[:3]))
        better += e1 < e0
        errs.append((round(float(e0), 4), round(float(e1), 4)))
        assert e1 < 0.05, errs
    assert better == 3, errs


def test_degenerate_cases(nv, room):
    """No correspondence (a scan far from the map) or fewer than six kept
    (a tiny tau): one linearization, not converged, the pose unchanged;
    bad voxel sizes are refused."""
    r, dt, keys, occ = room
    s, pose = synth.make_scan(1, 0)
    R0, t0 = _start(pose)
    far = nv.bbs_gicp(dt, s, R0, t0 + np.array([500.0, 0.0, 0.0]))
    assert far.status == nv.OK and far.correspondences == 0 and far.iterations == 1 and not far.converged
    Rg, tg = far.Rt()
    assert np.array_equal(Rg, R0) and np.array_equal(tg, t0 + np.array([500.0, 0.0, 0.0]))
    tiny = nv.bbs_gicp(dt, s[:20], R0, t0, nv.make_gicp_opts(tau=1e-6))
    o = gicp.gicp(occ, s[:20].astype(np.float64), R0, t0, r, tau=1e-6)
    assert tiny.correspondences == o.n < 6 and tiny.iterations == o.iterations == 1 and not tiny.converged
    for bad in (0.0, -1.0, float("nan")):
        with pytest.raises(nv.BBSError) as e:
            nv.bbs_gicp_target_build(synth.make_map(1)[:100], bad)
        assert e.value.code == nv.EINVAL

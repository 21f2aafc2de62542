"""Pins of the GICP refinement oracle (oracle/gicp.py): recovery of a known
transform, the Jacobian against finite differences, the normalized
covariance, the correspondence search against brute force, and the source
neighbourhoods against a k-d tree."""
import math

import numpy as np
import pytest

import oracle
from oracle import gicp
from paper_2310_10023_gb300 import synth


@pytest.fixture(scope="module")
def room_target():
    w = synth.WORKLOADS["room"]
    tgt = gicp.Target(synth.make_map(1), w.r)
    return tgt.r, tgt.keys, tgt


def _planted_scan(tgt, rng, n, R, t, noise=0.0):
    """Centroids of n occupied voxels, seen from pose (R, t): s = R^T (c - t)."""
    c = tgt.centroid[rng.choice(len(tgt.keys), n, replace=False)]
    s = (c - t) @ R        # rows: R^T (c - t)
    return (s + noise * rng.standard_normal(s.shape)).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_recovers_planted_transform(room_target, seed):
    """Voxel centres observed from a known pose: started 0.15 m and 0.03 rad
    off, GICP returns the pose (the residuals vanish there)."""
    r, keys, occ = room_target
    rng = np.random.default_rng(seed)
    R = gicp.rot_zyx(0.01, -0.015, 1.1 + seed)
    t = np.array([8.0 + seed, 9.5, 1.2])
    s = _planted_scan(occ, rng, 600, R, t)
    R0 = gicp.exp_so3(np.array([0.01, -0.01, 0.025])) @ R
    t0 = t + np.array([0.12, -0.08, 0.05])
    res = gicp.gicp(occ, s, R0, t0, r, max_iters=40)
    assert res.converged and res.iterations > 1
    assert np.linalg.norm(res.t - t) < 1e-4
    assert np.linalg.norm(res.R - R) < 1e-5
    assert res.cost < 1e-6


def test_jacobian_matches_finite_differences(room_target):
    r, keys, occ = room_target
    rng = np.random.default_rng(5)
    R = gicp.rot_zyx(0.0, 0.01, 0.4)
    t = np.array([10.0, 10.0, 1.0])
    s = _planted_scan(occ, rng, 300, R, t, noise=0.05)
    Cs = gicp.source_covariances(s, 2 * r, r, 1e-3)
    R1 = gicp.exp_so3(np.array([0.0, 0.0, 0.01])) @ R
    lin = gicp.linearize(occ, s, Cs, R1, t, r, r, 1e-3)
    # the cost with the correspondences and weights of this linearization held fixed
    p = gicp.transform(R1, t, s)
    idx = np.nonzero(lin.found)[0]
    c = occ.lookup(lin.voxels[idx])[1]
    M = np.linalg.inv(gicp.target_covariances(occ, lin.voxels[idx], r, 1e-3) + R1 @ Cs[idx] @ R1.T)

    def f(delta):
        q = p[idx] @ gicp.exp_so3(delta[:3]).T + delta[3:]
        d = c - q
        return float((d[:, None, :] @ M @ d[:, :, None]).sum())

    h = 1e-6
    num = np.array([(f(h * e) - f(-h * e)) / (2 * h) for e in np.eye(6)])
    assert np.allclose(num, 2 * lin.g, rtol=1e-5, atol=1e-6)
    assert abs(f(np.zeros(6)) - lin.cost) <= 1e-9 * max(1.0, lin.cost)
    assert np.allclose(lin.H, lin.H.T) and np.all(np.linalg.eigvalsh(lin.H) > 0)


def test_normalized_covariance(room_target):
    r, keys, occ = room_target
    eps = 1e-3
    C = gicp.target_covariances(occ, keys[:500], r, eps)
    tr = np.trace(C, axis1=1, axis2=2) / (r * r)
    iso = np.all(np.isclose(C, (r * r) * np.eye(3)), axis=(1, 2))
    assert np.allclose(tr[~iso], 1.0 + 3 * eps)
    assert np.allclose(C, np.transpose(C, (0, 2, 1)))
    assert np.all(np.linalg.eigvalsh(C) > 0)
    # an isolated voxel: r^2 I
    lone = gicp.Target(np.array([[0.1, 0.1, 0.1]], np.float32), r)
    assert np.allclose(gicp.target_covariances(lone, lone.keys, r, eps)[0], (r * r) * np.eye(3))
    # points along a line in x: the variance is all along x
    line = gicp.Target(np.array([[(i + 0.5) * r, 0.25 * r, 0.25 * r] for i in range(-3, 4)], np.float32), r)
    Cl = gicp.target_covariances(line, np.array([[0, 0, 0]]), r, eps)[0] / (r * r)
    assert np.allclose(Cl, np.diag([1 + eps, eps, eps]))


def test_centroids_are_exact_means(room_target):
    """The fixed-point centroid equals the FP64 mean of the voxel's points to
    within the 2^-32 m fixed-point step, and every point's key is its voxel's."""
    r, keys, tgt = room_target
    m = synth.make_map(1)
    u = gicp.fine_keys(m, r)
    sel = np.random.default_rng(2).choice(len(tgt.keys), 50, replace=False)
    for i in sel:
        pts = m[np.all(u == tgt.keys[i], axis=1)].astype(np.float64)
        assert len(pts) == tgt.count[i]
        assert np.allclose(tgt.centroid[i], pts.mean(axis=0), rtol=0, atol=1e-8)
        assert np.all(np.floor(tgt.centroid[i] / r + 1e-9) == tgt.keys[i])


def test_correspondence_equals_brute_force_within_half_voxel(room_target):
    """A centroid within half a voxel of p lies in the 3 x 3 x 3 block (it
    lies inside its voxel), so there the block search returns the global
    nearest centroid."""
    r, keys, occ = room_target
    rng = np.random.default_rng(9)
    sel = rng.choice(len(keys), 400, replace=False)
    p = occ.centroid[sel] + rng.uniform(-0.45, 0.45, (400, 3)) * r
    vox, cen, d2, found = gicp.correspondences(occ, p, r, r)
    checked = 0
    for i in range(len(p)):
        dd = ((p[i] - occ.centroid) ** 2).sum(axis=1)
        j = int(np.argmin(dd))
        if dd[j] <= (0.5 * r) ** 2:
            checked += 1
            assert found[i] and np.isclose(d2[i], dd[j], rtol=1e-12, atol=1e-15)
            assert tuple(vox[i]) == tuple(keys[j]) or np.isclose(dd[j], ((p[i] - cen[i]) ** 2).sum())
    assert checked > 100


def test_source_neighbourhoods_match_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(3)
    s = rng.uniform(-2.0, 2.0, (300, 3))
    rho, r, eps = 0.6, 0.5, 1e-3
    C = gicp.source_covariances(s, rho, r, eps)
    tree = spatial.cKDTree(s)
    for i in range(0, 300, 37):
        nb = s[tree.query_ball_point(s[i], rho * (1 + 1e-12))]
        S = np.cov(nb.T, bias=True) if len(nb) > 1 else np.zeros((3, 3))
        want = (r * r) * (S / np.trace(S) + eps * np.eye(3)) if np.trace(S) > 0 else (r * r) * np.eye(3)
        assert np.allclose(C[i], want, rtol=1e-9, atol=1e-12)


def test_pose_round_trip():
    pose = (1.0, -2.0, 3.0, 0.02, -0.03, 2.5)
    R, t = gicp.pose_to_rt(pose)
    assert np.allclose(gicp.rt_to_pose(R, t), pose)
    assert np.allclose(R @ R.T, np.eye(3))


def test_one_step_is_quadratic_near_the_solution(room_target):
    """From a pose 1e-3 off (rad and m) with every correspondence already the
    true one, one Gauss-Newton step on the linearization of the step's own
    parametrization (p -> Exp(w) p + v) lands within ~1e-5: the error
    shrinks quadratically, which an update inconsistent with that
    parametrization (e.g. t + v instead of Exp(w) t + v) does not achieve
    when t is metres from the origin."""
    r, keys, occ = room_target
    rng = np.random.default_rng(21)
    R = gicp.rot_zyx(0.0, 0.0, 0.3)
    t = np.array([12.0, 9.0, 1.0])
    s = _planted_scan(occ, rng, 500, R, t)
    R0 = gicp.exp_so3(np.array([0.0, 0.0, 1e-3])) @ R
    t0 = t + np.array([1e-3, -1e-3, 0.0])
    res = gicp.gicp(occ, s, R0, t0, r, max_iters=1)
    assert np.linalg.norm(res.t - t) < 2e-5
    assert np.linalg.norm(res.R - R) < 2e-6

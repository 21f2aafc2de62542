"""GICP refinement oracle (FP64, numpy): the local fine registration that
follows the branch-and-bound result (Sec. IV: the BnB estimate seeds a
generalized-ICP refinement).  Test infrastructure only -- imported by tests/
and bench.py's CPU legs, never by the product path.

The paper fixes none of GICP's internals; the readings here (shared with the
GPU path, each stated where it is used):

* Target: the map points grouped by fine voxel key u = floor(fl32(x fl32(1/r)))
  (the level-0 quantization of Sec. III-C); voxel u stands for the centroid of
  its points, u r + (sum_i rint((x_i - u r) 2^32)) 2^-32 / n, the sum taken
  in integers (exact, order-free), every other operation in FP64 rounded on
  its own.
* Correspondence of a transformed point p: among the occupied voxels of the
  3 x 3 x 3 block around floor(p / r), the one whose centroid is nearest
  (squared distance ((dx dx + dy dy) + dz dz), ties to the first in
  (dx, dy, dz) order, each offset from -1 to 1), kept when that distance is
  at most tau^2.
* Covariances, normalized and basis-free: C = r^2 (S / tr S + eps I) with S
  the (biased) sample covariance of the neighbourhood (target: the centroids
  of the occupied voxels of the 3 x 3 x 3 block around u; source: scan points
  within radius rho of the point); tr S = 0 gives C = r^2 I.  Sums run over
  neighbours in block or index order (the GPU sums the source neighbourhoods
  in a different fixed order: those covariances agree to FP64 rounding).
* Pose T = (R, t), R = Rz(yaw) Ry(pitch) Rx(roll); a step (w, v) maps p to
  Exp(w) p + v, so the residual d = c - p has Jacobian [ [p]_x | -I ];
  Gauss-Newton on sum_i d_i^T M_i d_i with M_i = (C_t + R C_s R^T)^-1 held
  fixed per linearization; stop when |w| < eps_rot and |v| < eps_trans
  (after applying the step) or after max_iters linearizations.
* Every transformed coordinate is ((R_i0 s_x + R_i1 s_y) + R_i2 s_z) + t_i,
  each operation rounded on its own, so both sides take the same voxel and
  correspondence decisions.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BIAS = 1 << 20


def pack_keys(v: np.ndarray) -> np.ndarray:
    """(n, 3) integer voxel keys -> int64 codes (21 bits per axis, offset 2^20)."""
    v = np.asarray(v, np.int64) + BIAS
    return (v[:, 0] << 42) | (v[:, 1] << 21) | v[:, 2]


FIX = float(1 << 32)


def fine_keys(xyz: np.ndarray, r: float) -> np.ndarray:
    """u = floor(fl32(x fl32(1/r))) per axis (the level-0 quantization)."""
    rho = np.float32(1.0 / r)
    return np.floor(np.asarray(xyz, np.float32) * rho).astype(np.int64)


class Target:
    """The map points grouped by fine voxel key, each voxel standing for the
    centroid of its points (fixed-point sums, exact)."""

    def __init__(self, xyz: np.ndarray, r: float):
        r = float(np.float32(r))   # the voxel size as the maps hold it (FP32)
        x = np.asarray(xyz, np.float32).reshape(-1, 3)
        u = fine_keys(x, r)
        codes, inv, cnt = np.unique(pack_keys(u), return_inverse=True, return_counts=True)
        rel = x.astype(np.float64) - u.astype(np.float64) * r
        fx = np.rint(rel * FIX).astype(np.int64)
        sums = np.zeros((len(codes), 3), np.int64)
        np.add.at(sums, inv, fx)
        first = np.zeros(len(codes), np.int64)
        first[inv[::-1]] = np.arange(len(x))[::-1]
        self.r = r
        self.codes = codes
        self.keys = u[first]
        self.count = cnt.astype(np.int64)
        self.centroid = self.keys.astype(np.float64) * r + (sums.astype(np.float64) / self.count[:, None]) / FIX

    def lookup(self, v: np.ndarray):
        """-> (found (n,) bool, centroid (n, 3)) for voxel keys v (n, 3)."""
        c = pack_keys(v)
        i = np.searchsorted(self.codes, c)
        i = np.minimum(i, max(len(self.codes) - 1, 0))
        hit = (self.codes[i] == c) if len(self.codes) else np.zeros(len(c), bool)
        return hit, np.where(hit[:, None], self.centroid[i] if len(self.codes) else 0.0, 0.0)


def rot_zyx(roll: float, pitch: float, yaw: float) -> np.ndarray:
    ca, sa = math.cos(roll), math.sin(roll)
    cb, sb = math.cos(pitch), math.sin(pitch)
    cg, sg = math.cos(yaw), math.sin(yaw)
    Rx = np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]])
    Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    Rz = np.array([[cg, -sg, 0], [sg, cg, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def pose_to_rt(pose) -> tuple:
    x, y, z, roll, pitch, yaw = pose
    return rot_zyx(roll, pitch, yaw), np.array([x, y, z], np.float64)


def rt_to_pose(R: np.ndarray, t: np.ndarray) -> tuple:
    yaw = math.atan2(R[1, 0], R[0, 0])
    pitch = -math.asin(max(-1.0, min(1.0, R[2, 0])))
    roll = math.atan2(R[2, 1], R[2, 2])
    return (float(t[0]), float(t[1]), float(t[2]), roll, pitch, yaw)


def transform(R: np.ndarray, t: np.ndarray, s: np.ndarray) -> np.ndarray:
    """p_i = ((R_i0 s_x + R_i1 s_y) + R_i2 s_z) + t_i, elementwise in FP64."""
    s = np.asarray(s, np.float64)
    out = np.empty_like(s)
    for i in range(3):
        out[:, i] = ((R[i, 0] * s[:, 0] + R[i, 1] * s[:, 1]) + R[i, 2] * s[:, 2]) + t[i]
    return out


def _normalized(S: np.ndarray, r: float, eps: float) -> np.ndarray:
    """r^2 (S / tr S + eps I), or r^2 I when tr S = 0; S (n, 6) as xx, xy, xz, yy, yz, zz."""
    tr = (S[:, 0] + S[:, 3]) + S[:, 5]
    C = np.zeros((len(S), 3, 3))
    idx = [(0, 0, 0), (1, 0, 1), (2, 0, 2), (3, 1, 1), (4, 1, 2), (5, 2, 2)]
    nz = tr > 0
    r2 = r * r
    for k, a, b in idx:
        val = np.where(nz, S[:, k] / np.where(nz, tr, 1.0), 0.0)
        if a == b:
            val = np.where(nz, val + eps, 1.0)
        C[:, a, b] = val * r2
        C[:, b, a] = val * r2
    return C


def target_covariances(tgt: Target, v: np.ndarray, r: float, eps: float) -> np.ndarray:
    """C_t of voxels v (n, 3): centroids of the occupied voxels of the 3 x 3 x 3 block."""
    v = np.asarray(v, np.int64)
    n = len(v)
    cnt = np.zeros(n)
    acc = np.zeros((n, 3))
    offs = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)]
    hits = []
    for dx, dy, dz in offs:
        h, c = tgt.lookup(v + np.array([dx, dy, dz]))
        hits.append((h, c))
        cnt += h
        acc += np.where(h[:, None], c, 0.0)
    den = np.maximum(cnt, 1.0)
    mu = acc / den[:, None]
    S = np.zeros((n, 6))
    for h, c in hits:
        ex = np.where(h, c[:, 0] - mu[:, 0], 0.0)
        ey = np.where(h, c[:, 1] - mu[:, 1], 0.0)
        ez = np.where(h, c[:, 2] - mu[:, 2], 0.0)
        S[:, 0] += ex * ex
        S[:, 1] += ex * ey
        S[:, 2] += ex * ez
        S[:, 3] += ey * ey
        S[:, 4] += ey * ez
        S[:, 5] += ez * ez
    S = S / den[:, None]
    return _normalized(S, r, eps)


def source_covariances(s: np.ndarray, rho: float, r: float, eps: float) -> np.ndarray:
    """C_s of every scan point: scan points within rho (FP64 distance, the point
    itself included), sums in index order."""
    s = np.asarray(s, np.float64)
    n = len(s)
    rho2 = rho * rho
    cnt = np.zeros(n)
    acc = np.zeros((n, 3))
    masks = []
    for j in range(n):
        dx = s[:, 0] - s[j, 0]
        dy = s[:, 1] - s[j, 1]
        dz = s[:, 2] - s[j, 2]
        m = ((dx * dx + dy * dy) + dz * dz) <= rho2
        masks.append(m)
        cnt += m
        acc += np.where(m[:, None], s[j], 0.0)
    mu = acc / cnt[:, None]
    S = np.zeros((n, 6))
    for j in range(n):
        m = masks[j]
        ex = np.where(m, s[j, 0] - mu[:, 0], 0.0)
        ey = np.where(m, s[j, 1] - mu[:, 1], 0.0)
        ez = np.where(m, s[j, 2] - mu[:, 2], 0.0)
        S[:, 0] += ex * ex
        S[:, 1] += ex * ey
        S[:, 2] += ex * ez
        S[:, 3] += ey * ey
        S[:, 4] += ey * ez
        S[:, 5] += ez * ez
    S = S / cnt[:, None]
    return _normalized(S, r, eps)


def correspondences(tgt: Target, p: np.ndarray, r: float, tau: float):
    """-> (voxel keys (n, 3), centroids (n, 3), squared distance (n,), found (n,) bool)."""
    p = np.asarray(p, np.float64)
    base = np.floor(p / r).astype(np.int64)
    n = len(p)
    best = np.full(n, np.inf)
    bv = np.zeros((n, 3), np.int64)
    bc = np.zeros((n, 3))
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                w = base + np.array([dx, dy, dz])
                h, c = tgt.lookup(w)
                ex, ey, ez = p[:, 0] - c[:, 0], p[:, 1] - c[:, 1], p[:, 2] - c[:, 2]
                d2 = (ex * ex + ey * ey) + ez * ez
                better = h & (d2 < best)
                best = np.where(better, d2, best)
                bv = np.where(better[:, None], w, bv)
                bc = np.where(better[:, None], c, bc)
    found = best <= tau * tau
    return bv, bc, best, found


def skew(p: np.ndarray) -> np.ndarray:
    K = np.zeros(p.shape[:-1] + (3, 3))
    K[..., 0, 1], K[..., 0, 2] = -p[..., 2], p[..., 1]
    K[..., 1, 0], K[..., 1, 2] = p[..., 2], -p[..., 0]
    K[..., 2, 0], K[..., 2, 1] = -p[..., 1], p[..., 0]
    return K


@dataclass
class Linearization:
    H: np.ndarray        # 6 x 6
    g: np.ndarray        # 6
    cost: float
    n: int               # correspondences kept
    voxels: np.ndarray   # per point: the target voxel (undefined where not found)
    found: np.ndarray


def linearize(tgt: Target, s: np.ndarray, Cs: np.ndarray, R: np.ndarray, t: np.ndarray, r: float, tau: float,
              eps: float) -> Linearization:
    p = transform(R, t, s)
    vox, cen, _, found = correspondences(tgt, p, r, tau)
    H = np.zeros((6, 6))
    g = np.zeros(6)
    cost = 0.0
    idx = np.nonzero(found)[0]
    if len(idx):
        pk = p[idx]
        d = cen[idx] - pk
        Ct = target_covariances(tgt, vox[idx], r, eps)
        C = Ct + R @ Cs[idx] @ R.T
        M = np.linalg.inv(C)
        J = np.concatenate([skew(pk), -np.broadcast_to(np.eye(3), (len(idx), 3, 3))], axis=2)   # (n, 3, 6)
        JtM = np.transpose(J, (0, 2, 1)) @ M
        H = (JtM @ J).sum(axis=0)
        g = (JtM @ d[:, :, None])[:, :, 0].sum(axis=0)
        cost = float((d[:, None, :] @ M @ d[:, :, None]).sum())
    return Linearization(H, g, cost, int(len(idx)), vox, found)


def exp_so3(w: np.ndarray) -> np.ndarray:
    th = float(np.linalg.norm(w))
    K = skew(np.asarray(w, np.float64))
    if th < 1e-12:
        return np.eye(3) + K
    return np.eye(3) + (math.sin(th) / th) * K + ((1.0 - math.cos(th)) / (th * th)) * (K @ K)


@dataclass
class GicpResult:
    R: np.ndarray
    t: np.ndarray
    iterations: int
    cost: float
    n: int
    converged: bool


def gicp(tgt: Target, s: np.ndarray, R0: np.ndarray, t0: np.ndarray, r: float, tau: float | None = None,
         rho: float | None = None, eps: float = 1e-3, max_iters: int = 30, eps_rot: float = 1e-6,
         eps_trans: float = 1e-6) -> GicpResult:
    tau = r if tau is None else tau
    rho = 2.0 * r if rho is None else rho
    Cs = source_covariances(s, rho, r, eps)
    R, t = np.array(R0, np.float64), np.array(t0, np.float64)
    lin = None
    for it in range(1, max_iters + 1):
        lin = linearize(tgt, s, Cs, R, t, r, tau, eps)
        if lin.n < 6:
            return GicpResult(R, t, it, lin.cost, lin.n, False)
        delta = np.linalg.solve(lin.H, -lin.g)
        w, v = delta[:3], delta[3:]
        E = exp_so3(w)
        R = E @ R
        t = E @ t + v
        if np.linalg.norm(w) < eps_rot and np.linalg.norm(v) < eps_trans:
            return GicpResult(R, t, it, lin.cost, lin.n, True)
    return GicpResult(R, t, max_iters, lin.cost if lin else 0.0, lin.n if lin else 0, False)

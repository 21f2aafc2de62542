"""Pins of the oracle's pose grid (Sec. III-B Eq. (2)-(5), Sec. III-D Eq. (12)-(14))
against closed forms, an independent rotation library and structural invariants."""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_delta_closed_forms():
    cases = json.load(open(os.path.join(GOLD, "delta_closed_forms.json")))["cases"]
    for c in cases:
        for d in (0.5, 7.0, 123.0):
            got = oracle.delta(c["r_over_dmax"] * d, d)
            assert abs(got - c["delta"]) <= 4e-15 * max(1.0, c["delta"]) * 4, (c, d, got)


@pytest.mark.parametrize("r,d", [(0.2, 50.0), (0.5, 24.5), (1.0, 100.0), (3.2, 50.0), (64.0, 40.0)])
def test_delta_chord_identity(r, d):
    # a point at range d_max moves by exactly r under a rotation of delta(r):
    # chord length 2 d_max sin(delta / 2) = r  (Eq. (2) rewritten)
    dl = oracle.delta(r, d)
    assert abs(2 * d * math.sin(dl / 2) - r) <= 1e-12 * r


def test_delta_degenerate():
    assert oracle.delta(1.0, 0.0) == pytest.approx(math.pi)
    assert oracle.delta(10.0, 1.0) == pytest.approx(math.pi)


def _grid(r=0.5, levels=4, dmax=24.5, ang=((-0.05, 0.05), (-0.05, 0.05), (0.0, 2 * math.pi)),
          lo=(0, 0, 0), hi=(20, 20, 5), flags=0):
    rg = oracle.make_ranges(lo, hi, [a[0] for a in ang], [a[1] for a in ang])
    return oracle.Grid(r, levels, dmax, rg, flags), rg


@pytest.mark.parametrize("dmax", [5.0, 24.5, 51.3, 99.0])
def test_grid_segments(dmax):
    g, _ = _grid(r=0.2, levels=7, dmax=dmax)
    for l in range(g.levels):
        rl = 0.2 * 2 ** l
        dl = oracle.delta(np.float32(0.2) * 2.0 ** l, dmax)
        assert g.delta(l) == dl
        for ax, W in enumerate((0.1, 0.1, 2 * math.pi)):
            n = g.N(l)[ax]
            # Eq. (12): N = ceil(W / delta), delta' = W / N <= delta, N delta' = W
            assert n == max(1, math.ceil(W / dl))
            assert g.dprime(l)[ax] <= dl * (1 + 1e-15)
            assert abs(n * g.dprime(l)[ax] - W) <= 1e-15 * W * 4
        del rl
    for l in range(1, g.levels):
        for ax in range(3):
            np_, nc = g.N(l)[ax], g.N(l - 1)[ax]
            a = g.a(l)[ax]
            # Eq. (14) with delta'_l / delta'_{l-1} = N_{l-1} / N_l exactly
            assert a == (1 if nc <= 1 else math.ceil(nc / np_))
            assert a * np_ >= nc


@pytest.mark.parametrize("dmax", [5.0, 24.5, 51.3])
def test_children_partition_and_nesting(dmax):
    """Every level-(l-1) angle index has exactly one parent, no parent has more than
    a children, and each child's angle lies inside its parent's segment."""
    g, _ = _grid(r=0.2, levels=6, dmax=dmax)
    for l in range(1, g.levels):
        for ax in range(3):
            np_, nc = g.N(l)[ax], g.N(l - 1)[ax]
            owner = np.full(nc, -1)
            for c in range(np_):
                node = [0, 0, 0, 0, 0, 0, l]
                node[3 + ax] = c
                kids = g.children(node)
                idx = sorted(set(int(k[3 + ax]) for k in kids))
                assert len(idx) <= g.a(l)[ax]
                for ci in idx:
                    assert owner[ci] == -1
                    owner[ci] = c
                    lo_edge = g.angle(l, ax, c) - g.dprime(l)[ax] / 2
                    hi_edge = g.angle(l, ax, c) + g.dprime(l)[ax] / 2
                    ang = g.angle(l - 1, ax, ci)
                    assert lo_edge - 1e-12 <= ang <= hi_edge + 1e-12
            assert (owner >= 0).all()


def test_children_match_eq13_when_grids_nest():
    # wherever N_{l-1} = a N_l exactly, the children are a*c + j, j < a (Eq. (13))
    checked = 0
    for dmax in (3.0, 7.5, 12.0, 24.5, 40.0, 51.3):
        g, _ = _grid(r=0.5, levels=5, dmax=dmax, ang=((-0.1, 0.1), (-0.05, 0.05), (0.0, 2 * math.pi)))
        for l in range(1, 5):
            for ax in range(3):
                np_, nc = g.N(l)[ax], g.N(l - 1)[ax]
                if nc % np_ != 0 or nc == np_:
                    continue
                a = nc // np_
                checked += 1
                for c in range(np_):
                    node = [0, 0, 0, 0, 0, 0, l]
                    node[3 + ax] = c
                    got = sorted(set(int(k[3 + ax]) for k in g.children(node)))
                    assert got == [a * c + j for j in range(a)]
    assert checked > 0


def test_children_translations_and_count():
    g, _ = _grid(r=0.5, levels=3, dmax=24.5)
    p = [3, -2, 1, 1, 0, 40, 2]
    kids = g.children(p)
    assert len(kids) == g.num_children(p)
    trans = set(tuple(k[:3]) for k in kids)
    assert trans == {(6 + jx, -4 + jy, 2 + jz) for jx in (0, 1) for jy in (0, 1) for jz in (0, 1)}
    assert all(k[6] == 1 for k in kids)
    assert g.num_children([0, 0, 0, 0, 0, 0, 0]) == 0


def test_child_literal_flag_is_eq13_verbatim():
    g, _ = _grid(r=0.5, levels=3, dmax=24.5, flags=oracle.CHILD_LITERAL)
    for l in (1, 2):
        a = g.a(l)
        for c in range(g.N(l)[2]):
            got = sorted(set(int(k[5]) for k in g.children([0, 0, 0, 0, 0, c, l])))
            want = [a[2] * c + j for j in range(a[2]) if a[2] * c + j < g.N(l - 1)[2]]
            assert got == want


def test_initial_translation_bounds():
    # Eq. (3)-(5): w_min = floor(W_min / (2^lmax r)), w_max = ceil(W_max / (2^lmax r))
    g, _ = _grid(r=0.5, levels=3, lo=(-3.1, 0.0, 0.5), hi=(20.0, 7.9, 5.0))
    (a0, a1, a2), (b0, b1, b2) = g.wrange()
    assert (a0, a1, a2) == (math.floor(-3.1 / 2), 0, math.floor(0.5 / 2))
    assert (b0, b1, b2) == (10, math.ceil(7.9 / 2), math.ceil(5.0 / 2))


def test_translation_only_grid():
    g, _ = _grid(r=0.5, levels=4, flags=oracle.TRANSLATION_ONLY)
    for l in range(4):
        assert g.N(l) == g.N(0)
        assert g.delta(l) == g.delta(0)
    for l in range(1, 4):
        assert g.a(l) == (1, 1, 1)


def test_angles_segment_centre_and_lower_edge():
    g, _ = _grid()
    g2, _ = _grid(flags=oracle.ANGLE_LOWER_EDGE)
    for l in range(3):
        dp = g.dprime(l)[2]
        assert g.angle(l, 2, 0) == pytest.approx(dp / 2, rel=1e-15)
        assert g2.angle(l, 2, 0) == 0.0
        n = g.N(l)[2]
        assert g.angle(l, 2, n - 1) == pytest.approx(2 * math.pi - dp / 2, rel=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_rotation_against_scipy(seed):
    """A = fl32(R / r) with R = Rz(yaw) Ry(pitch) Rx(roll): compared with an
    independent Euler-angle implementation (intrinsic 'ZYX' = yaw, pitch, roll)."""
    rng = np.random.default_rng(seed)
    r = float(np.float32(rng.uniform(0.1, 2.0)))
    g, _ = _grid(r=r, levels=3, dmax=30.0, ang=((-0.3, 0.3), (-0.2, 0.25), (0.0, 2 * math.pi)))
    for _ in range(50):
        l = int(rng.integers(0, 3))
        ia, ib, ig = (int(rng.integers(0, g.N(l)[i])) for i in range(3))
        roll, pitch, yaw = g.angle(l, 0, ia), g.angle(l, 1, ib), g.angle(l, 2, ig)
        R = Rotation.from_euler("ZYX", [yaw, pitch, roll]).as_matrix()
        A = g.rotation(l, ia, ib, ig).astype(np.float64).reshape(3, 3)
        ref = R / r
        # the oracle rounds its own FP64 product once to FP32: within 1 ulp
        # of FP32 plus the FP64 difference between two evaluation orders
        ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(A - ref) <= ulp * 1.01 + 1e-12), (A, ref)


def test_rotation_identity_and_orthonormal():
    g, _ = _grid(r=1.0, levels=1, dmax=30.0, ang=((0, 0), (0, 0), (0, 0)))
    A = g.rotation(0, 0, 0, 0).reshape(3, 3)
    assert np.array_equal(A, np.eye(3, dtype=np.float32))
    g, _ = _grid(r=1.0, levels=2, dmax=30.0)
    for ig in range(0, g.N(0)[2], 17):
        A = g.rotation(0, 1, 2, ig).astype(np.float64).reshape(3, 3)
        assert np.allclose(A @ A.T, np.eye(3), atol=1e-6)
        assert np.linalg.det(A) == pytest.approx(1.0, abs=1e-6)


def test_grid_rejects_bad_input():
    rg = oracle.make_ranges((0, 0, 0), (1, 1, 1), (0, 0, 0), (0, 0, 1))
    with pytest.raises(ValueError):
        oracle.Grid(-1.0, 3, 10.0, rg)
    with pytest.raises(ValueError):
        oracle.Grid(0.5, 0, 10.0, rg)
    with pytest.raises(ValueError):
        oracle.Grid(0.5, 17, 10.0, rg)
    bad = oracle.make_ranges((0, 0, 0), (1, 1, 1), (0, 0, 1), (0, 0, 0))
    with pytest.raises(ValueError):
        oracle.Grid(0.5, 3, 10.0, bad)
    far = oracle.make_ranges((0, 0, 0), (1e6, 1, 1), (0, 0, 0), (0, 0, 1))
    with pytest.raises(ValueError):
        oracle.Grid(0.5, 3, 10.0, far)   # leaf translations beyond +-2^20 voxels

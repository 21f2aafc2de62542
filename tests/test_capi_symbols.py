"""The C-ABI library loads and exports every function include/bbs.h declares
(no compute call: this runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bbs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(bbs_[a-z_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2310_10023_gb300 import build, native
    build.build()
    lib = native.load()
    declared = _declared()
    assert {"bbs_build_maps", "bbs_localize", "bbs_score_batch"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_function():
    from paper_2310_10023_gb300 import native
    for n in _declared():
        assert hasattr(native, n), n


def test_version_string():
    from paper_2310_10023_gb300 import native
    assert "sm_103a" in native.bbs_version()


def test_tuning_validation_without_gpu():
    """bbs_set_tuning checks its ranges on the host (no device work)."""
    from paper_2310_10023_gb300 import native as nv
    nv.load()
    for bad in ({"launch_tasks": (1 << 19) + 1}, {"static_pm": 1001}, {"grab_min": -3}, {"ctas_per_sm": 5}):
        with pytest.raises(nv.BBSError) as e:
            nv.bbs_set_tuning(**bad)
        assert e.value.code == nv.EINVAL
    nv.bbs_set_tuning(launch_tasks=100, static_pm=500)
    assert nv.bbs_get_tuning() == {"launch_tasks": 100, "static_pm": 500, "grab_min": 16, "ctas_per_sm": 4,
                                   "frontier_log2": 0}
    nv.bbs_set_tuning(reset=True)
    assert nv.bbs_get_tuning()["launch_tasks"] == 1 << 19


def test_layout_and_load_validation_without_gpu():
    """bbs_set_probe_layout and bbs_set_load_factor check their ranges on the host."""
    from paper_2310_10023_gb300 import native as nv
    nv.load()
    for bad in (-1, 5):
        with pytest.raises(nv.BBSError) as e:
            nv.bbs_set_probe_layout(bad)
        assert e.value.code == nv.EINVAL
    for bad in (0.0, 0.01, 0.95, float("nan")):
        with pytest.raises(nv.BBSError) as e:
            nv.bbs_set_load_factor(bad)
        assert e.value.code == nv.EINVAL
    for ok in (1, 2, 3, 4, 0):
        nv.bbs_set_probe_layout(ok)
    nv.bbs_set_load_factor(0.25)


def test_server_slot_limit_without_gpu():
    """A server advances at most 256 searches together (the search id is the
    top byte of a frontier key): a larger max_active is refused on the host."""
    from paper_2310_10023_gb300 import native as nv
    nv.load()
    with pytest.raises(nv.BBSError) as e:
        nv.bbs_server_create(max_active=257)
    assert e.value.code == nv.EINVAL
    assert "256" in nv.bbs_last_error()


def test_pose_matrix_is_intrinsic_zyx_euler_without_gpu():
    """bbs_pose_matrix (host code in the library) composes R = Rz(yaw)
    Ry(pitch) Rx(roll), Sec. III-A's angles; pinned against scipy's
    intrinsic ZYX Euler rotation, an independent construction that catches a
    wrong order, sign or transpose."""
    Rotation = pytest.importorskip("scipy.spatial.transform").Rotation
    import numpy as np
    from paper_2310_10023_gb300 import native as nv
    nv.load()
    rng = np.random.default_rng(5)
    for _ in range(50):
        pose = np.concatenate([rng.uniform(-50, 50, 3), rng.uniform(-np.pi, np.pi, 3)])
        R, t = nv.bbs_pose_matrix(pose)
        want = Rotation.from_euler("ZYX", [pose[5], pose[4], pose[3]]).as_matrix()
        assert np.allclose(R, want, atol=1e-14)
        assert np.array_equal(t, pose[:3])
    with pytest.raises(nv.BBSError) as e:
        nv.bbs_pose_matrix([0, 0, 0, float("nan"), 0, 0])
    assert e.value.code == nv.EINVAL

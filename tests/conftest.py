import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def room():
    """Room workload (20 x 20 x 5 m, r = 0.5 m, 3 levels) with its first scan."""
    from paper_2310_10023_gb300 import synth
    w = synth.WORKLOADS["room"]
    m = synth.make_map(w.scene)
    s, pose = synth.make_scan(w.scene, 0)
    return w, m, s, pose


@pytest.fixture(scope="session")
def room_oracle_maps(room):
    import oracle
    w, m, _, _ = room
    return oracle.Maps(m, w.r, w.levels)

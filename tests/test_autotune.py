"""The launch-shape autotuner: its cache (CPU) and one tuning run that keeps
every result unchanged (GPU)."""
import os

import pytest

from paper_2310_10023_gb300 import autotune, synth


def test_cache_key_and_store(tmp_path):
    k1 = autotune.workload_key("GB300", 152, 0.2, 6, 16384, [2100, 30000])
    k2 = autotune.workload_key("GB300", 152, 0.2, 6, 16384, [2200, 31000])   # same log2 buckets
    k3 = autotune.workload_key("GB300", 152, 1.0, 8, 16384, [2000, 30000])
    assert k1 == k2 and k1 != k3 and k1.startswith("GB300|152|")
    p = str(tmp_path / "t.json")
    assert autotune.load_cache(p) == {}
    autotune.store(k1, {"best": dict(autotune.DEFAULT), "ms": 1.0, "trials": []}, p)
    autotune.store(k3, {"best": dict(autotune.DEFAULT, static_pm=500), "ms": 2.0, "trials": []}, p)
    data = autotune.load_cache(p)
    assert data[k1]["ms"] == 1.0 and data[k3]["best"]["static_pm"] == 500


@pytest.mark.gpu
def test_autotune_keeps_results(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_10023_gb300 import build, native as nv
    build.build()
    nv.load()
    w = synth.WORKLOADS["room"]
    m = synth.make_map(w.scene)
    scans = [torch.from_numpy(synth.make_scan(w.scene, i)[0]).cuda() for i in range(2)]
    rg = nv.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    op = nv.make_opts(score_frac=w.score_frac, batch=w.batch)
    p = str(tmp_path / "tuning.json")
    space = {"layout": [0, 2], "load_factor": [0.5, 0.25], "static_pm": [500, 750], "ctas_per_sm": [3, 4]}
    try:
        out = autotune.tuned("gpu", 1, lambda: nv.bbs_build_maps(m, w.r, w.levels), scans, rg, op, w.r, w.levels,
                             [len(s) for s in scans], path=p, reps=1, space=space)
        assert not out["cached"] and len(out["trials"]) >= 3 and os.path.exists(p)
        again = autotune.tuned("gpu", 1, None, scans, rg, op, w.r, w.levels, [len(s) for s in scans], path=p)
        assert again["cached"] and again["best"] == out["best"]
    finally:
        nv.bbs_set_tuning(reset=True)
        nv.bbs_set_load_factor(0.25)
        nv.bbs_set_probe_layout(0)

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


def test_batch_search_keeps_the_best_score():
    """search_batch takes the fastest batch among those that keep every
    scan's best score (a faster batch that loses a point is refused)."""
    from types import SimpleNamespace

    from paper_2310_10023_gb300 import native as nv
    # scripted searches: per batch, (best scores of the two scans, ms per localization)
    script = {16384: ([950, 960], 1.0), 4096: ([950, 960], 0.9), 8192: ([950, 959], 0.5),
              32768: ([950, 960], 0.8), 65536: ([950, 960], 1.2)}
    clock = {"t": 0.0}

    def localize(maps, scan, ranges, o):
        scores, ms = script[int(o.batch)]
        clock["t"] += ms / 1e3
        return SimpleNamespace(best_score=scores[scan], nodes_scored=int(o.batch))

    opts = nv.make_opts(batch=16384, stream=0)
    out = autotune.search_batch(None, [0, 1], None, opts, reps=2, timer=lambda: clock["t"], sync=lambda: None,
                                localize=localize)
    assert out["batch"] == 32768                                  # 8192 is faster but changes a score
    by_b = {t["batch"]: t for t in out["trials"]}
    assert not by_b[8192]["accepted"] and by_b[4096]["accepted"] and by_b[65536]["accepted"]
    assert by_b[16384]["ms"] == pytest.approx(2.0) and out["ms"] == pytest.approx(1.6)
    assert opts.batch == 16384                                    # the caller's options are left alone


@pytest.mark.gpu
def test_tuned_batch_keeps_best_scores(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_10023_gb300 import build, native as nv
    build.build()
    nv.load()
    w = synth.WORKLOADS["room"]
    m = synth.make_map(w.scene)
    scans = [torch.from_numpy(synth.make_scan(w.scene, i)[0]).cuda() for i in range(3)]
    rg = nv.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    op = nv.make_opts(score_frac=w.score_frac, batch=w.batch)
    p = str(tmp_path / "tuning.json")
    try:
        out = autotune.tuned("gpu", 1, lambda: nv.bbs_build_maps(m, w.r, w.levels), scans, rg, op, w.r, w.levels,
                             [len(s) for s in scans], path=p, reps=1, space={"static_pm": [500]}, tune_batch=True)
        assert out["batch"] in set(autotune.BATCHES) | {w.batch}
        assert {t["batch"] for t in out["batch_trials"]} == set(autotune.BATCHES) | {w.batch}
        dm = nv.bbs_build_maps(m, w.r, w.levels)
        ref = [nv.bbs_localize(dm, s, rg, op).best_score for s in scans]
        tb = nv.make_opts(score_frac=w.score_frac, batch=out["batch"])
        assert [nv.bbs_localize(dm, s, rg, tb).best_score for s in scans] == ref
        again = autotune.tuned("gpu", 1, None, scans, rg, op, w.r, w.levels, [len(s) for s in scans], path=p,
                               tune_batch=True)
        assert again["cached"] and again["batch"] == out["batch"]
    finally:
        nv.bbs_set_tuning(reset=True)
        nv.bbs_set_load_factor(0.25)
        nv.bbs_set_probe_layout(0)

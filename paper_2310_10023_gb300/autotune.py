"""Launch-shape autotuner for the batched search (the tile / layout choices
of the scoring path), with a JSON cache keyed by GPU and workload shape.

What is tuned never changes a result: the level maps' layout (byte grids
where a level's box allows, or hashed bricks everywhere), the load factor of
the hashed tables (probe length vs footprint; byte grids have none), the
share of a scoring launch split statically over the CTAs, the smallest
dynamic grab, and the scoring CTAs per SM.  Every candidate's results are
compared with the first candidate's; a candidate that differs is an error.

The node batch b is tuned only on request (search_batch, tuned(...,
tune_batch=True)): b is part of the search's definition (it changes the
trajectory, Algorithm 2) and, under the approximate rotational bound, can
change the best score found.  A candidate b is accepted only when every
tuning scan reaches the same best score as with the caller's b; the fastest
accepted b is kept.

Coordinate descent: each knob in turn, the others held at their best so far;
the time of a candidate is the median over `reps` passes of bbs_localize on
the given device-resident scans.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
import time

from . import native as nv

DEFAULT = {"layout": 0, "load_factor": 0.25, "static_pm": 750, "grab_min": 16, "ctas_per_sm": 4}
SPACE = {
    "layout": [0, 2],
    "load_factor": [0.5, 0.35, 0.25, 0.15],
    "static_pm": [625, 750, 1000],
    "grab_min": [8, 16, 32],
    "ctas_per_sm": [3, 4],
}


def cache_path() -> str:
    p = os.environ.get("BBS_TUNING_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2310_10023_gb300", "tuning.json")


def workload_key(gpu: str, sms: int, r: float, levels: int, batch: int, ks) -> str:
    """GPU name and SM count, voxel size, levels, batch and the scan-size
    range (log2 buckets): tunings transfer between workloads of one shape."""
    kmin, kmax = min(ks), max(ks)
    shape = f"r={r:.6g};L={levels};b={batch};k={kmin.bit_length()}-{kmax.bit_length()}"
    return f"{gpu}|{sms}|{hashlib.sha1(shape.encode()).hexdigest()[:12]}|{shape}"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store(key: str, entry: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    data = load_cache(path)
    data[key] = entry
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(cfg: dict) -> None:
    """Make cfg the library's launch shape, map layout and load factor (maps
    built after this call use the layout and the load factor)."""
    nv.bbs_set_probe_layout(int(cfg.get("layout", DEFAULT["layout"])))
    nv.bbs_set_load_factor(float(cfg.get("load_factor", DEFAULT["load_factor"])))
    nv.bbs_set_tuning(static_pm=int(cfg.get("static_pm", DEFAULT["static_pm"])),
                      grab_min=int(cfg.get("grab_min", DEFAULT["grab_min"])),
                      ctas_per_sm=int(cfg.get("ctas_per_sm", DEFAULT["ctas_per_sm"])))


def _result_key(r) -> tuple:
    return (r.status, r.best_score, tuple(r.node), r.iterations, r.nodes_scored)


def search(build_maps, scans, ranges, opts, reps: int = 3, space: dict | None = None, timer=None,
           sync=None) -> dict:
    """Coordinate descent over `space` (default SPACE).

    build_maps() -> maps handle (called again whenever the layout or the
    load factor changes); scans: device-resident point arrays; timer/sync: clock and
    device synchronization (defaults: time.perf_counter and
    torch.cuda.synchronize).  Returns {"best": cfg, "ms": per-pass ms,
    "trials": [...]}.
    """
    space = space or SPACE
    if sync is None:
        import torch
        sync = torch.cuda.synchronize
    timer = timer or time.perf_counter
    best = dict(DEFAULT)
    ref = None
    trials = []
    maps_cache = {}

    def maps_for(layout, lf):
        if (layout, lf) not in maps_cache:
            nv.bbs_set_probe_layout(layout)
            nv.bbs_set_load_factor(lf)
            maps_cache[(layout, lf)] = build_maps()
        return maps_cache[(layout, lf)]

    def run(cfg):
        nonlocal ref
        apply(cfg)
        m = maps_for(cfg.get("layout", DEFAULT["layout"]), cfg["load_factor"])
        keys = [_result_key(nv.bbs_localize(m, s, ranges, opts)) for s in scans]   # warm-up + check
        if ref is None:
            ref = keys
        elif keys != ref:
            raise RuntimeError(f"autotune: launch shape {cfg} changed a result")
        times = []
        for _ in range(reps):
            sync()
            t = timer()
            for s in scans:
                nv.bbs_localize(m, s, ranges, opts)
            sync()
            times.append((timer() - t) * 1e3)
        ms = statistics.median(times)
        trials.append({"cfg": dict(cfg), "ms": ms})
        return ms

    best_ms = run(best)
    for knob, values in space.items():
        for v in values:
            if v == best[knob]:
                continue
            cand = dict(best, **{knob: v})
            ms = run(cand)
            if ms < best_ms:
                best, best_ms = cand, ms
    apply(best)
    return {"best": best, "ms": best_ms, "trials": trials}


BATCHES = (4096, 8192, 16384, 32768, 65536)   # the node batches the workloads allow


def search_batch(maps, scans, ranges, opts, batches=BATCHES, reps: int = 3, timer=None, sync=None,
                 localize=None) -> dict:
    """The fastest node batch b among `batches` that keeps every scan's best
    score equal to the one reached with opts.batch (the reference).

    Time of a candidate: the median over `reps` passes of localizing every
    scan.  Returns {"batch": b, "ms": per-pass ms, "trials": [{"batch", "ms",
    "best_scores", "nodes_scored", "accepted"}]}; with no accepted candidate
    faster than the reference, the reference b.
    """
    if sync is None:
        import torch
        sync = torch.cuda.synchronize
    timer = timer or time.perf_counter
    localize = localize or nv.bbs_localize
    ref_b = int(opts.batch)
    trials = []

    def run(b):
        o = nv.Opts.from_buffer_copy(opts)   # the caller's options, this batch
        o.batch = int(b)
        res = [localize(maps, s, ranges, o) for s in scans]   # warm-up, and the scores compared
        times = []
        for _ in range(reps):
            sync()
            t = timer()
            for s in scans:
                localize(maps, s, ranges, o)
            sync()
            times.append((timer() - t) * 1e3)
        return statistics.median(times), [r.best_score for r in res], sum(int(r.nodes_scored) for r in res)

    ref_ms, ref_scores, ref_nodes = run(ref_b)
    trials.append({"batch": ref_b, "ms": ref_ms, "best_scores": ref_scores, "nodes_scored": ref_nodes,
                   "accepted": True})
    best_b, best_ms = ref_b, ref_ms
    for b in batches:
        if int(b) == ref_b:
            continue
        ms, scores, nodes = run(b)
        ok = scores == ref_scores
        trials.append({"batch": int(b), "ms": ms, "best_scores": scores, "nodes_scored": nodes, "accepted": ok})
        if ok and ms < best_ms:
            best_b, best_ms = int(b), ms
    return {"batch": best_b, "ms": best_ms, "trials": trials}


def tuned(gpu: str, sms: int, build_maps, scans, ranges, opts, r: float, levels: int, ks, path: str | None = None,
          tune_batch: bool = False, **kw) -> dict:
    """The cached launch shape for this GPU and workload shape, searched and
    stored on a miss; applied before returning.  With tune_batch, the entry
    also holds the node batch search_batch picked ("batch"; the caller sets
    it in its options)."""
    key = workload_key(gpu, sms, r, levels, int(opts.batch), ks) + (";tuned-b" if tune_batch else "")
    hit = load_cache(path).get(key)
    if hit is not None:
        apply(hit["best"])
        return dict(hit, cached=True)
    out = search(build_maps, scans, ranges, opts, **kw)
    entry = {"best": out["best"], "ms": out["ms"], "trials": out["trials"]}
    if tune_batch:
        m = build_maps()
        bt = search_batch(m, scans, ranges, opts, reps=kw.get("reps", 3), timer=kw.get("timer"),
                          sync=kw.get("sync"))
        entry.update(batch=bt["batch"], batch_ms=bt["ms"], batch_trials=bt["trials"])
    store(key, entry, path)
    return dict(entry, cached=False)

"""Run independent oracle searches side by side on the host's cores (test
helper).  The pool uses the spawn start method, so it is safe after CUDA has
been initialized in the calling process; each worker builds the oracle maps
of a workload once."""
import multiprocessing as mp
import os

_MAPS = {}


def _maps(name, flags):
    import oracle
    from paper_2310_10023_gb300 import synth
    key = (name, flags)
    if key not in _MAPS:
        w = synth.WORKLOADS[name]
        _MAPS[key] = oracle.Maps(synth.make_map(w.scene), w.r, w.levels, flags)
    return _MAPS[key]


def _job(args):
    import oracle
    name, scan, ranges, score_frac, batch, flags, map_flags = args
    om = _maps(name, map_flags)
    rg = oracle.make_ranges(*ranges)
    r = oracle.localize(om, scan, rg, score_frac=score_frac, batch=batch, flags=flags)
    return {k: (list(getattr(r, k)) if k in ("node", "pose") else getattr(r, k))
            for k in ("status", "best_score", "node", "pose", "iterations", "nodes_scored", "peak_frontier",
                      "children_scored", "bound_violations", "bound_excess")}


def localize_many(jobs, procs=None):
    """jobs: (workload name, scan (k, 3) float32, (lo, hi, ang_lo, ang_hi),
    score_frac, batch, flags, map_flags) -> one result dict per job."""
    procs = procs or max(1, min(len(jobs), (os.cpu_count() or 2) - 1))
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        return pool.map(_job, jobs, chunksize=1)

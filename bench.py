"""Benchmark: candidate-pose point-probes/s and ms-to-optimum of GPU 3D-BBS.

One step = one global localization (bbs_localize through the C-ABI) of one
synthetic scan against the resident indoor map: 100 x 60 x 10 m multi-room
floor, ~5 M map points, r = 0.2 m, 6 levels, 16-beam scans of ~8 k points.
Scans cycle through a fixed set; each rank localizes its own scans (replicas:
the maps are rebuilt per GPU and no data crosses GPUs).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`value` is point-probes (children scored x scan points) per second over the
timed steps with the scan already in HBM; `e2e` repeats the steps through the
same C-ABI call with host buffers (scan H2D and result D2H inside the timed
region).  The reference arm times the CPU oracle on a bounded node sample.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "candidate-pose point-probes/sec and ms-to-optimum per scan (batched vs plain, same GPU)"
# Algorithmic work of Eq. (11): per probe (one scan point x one rotational
# child, which answers its 8 translational children) 3 translation adds and
# 8 child counts; per rotated scan point 9 products, 6 sums and 3 floors
# (with the level shift) -- once per point for all tasks that share a rotation
OPS_PER_PROBE = 11
OPS_PER_ROTATION = 18
WORKLOAD = "indoor"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=24)
    p.add_argument("--warmup", type=int, default=4)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--scans", type=int, default=8, help="distinct scans cycled by the steps")
    p.add_argument("--workload", choices=["indoor", "outdoor"], default=WORKLOAD,
                   help="the workload of the timed steps (indoor: the headline configuration)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip the batched and served forms")
    p.add_argument("--autotune", action="store_true",
                   help="choose the launch shape and table load with the autotuner (cached per GPU and workload)")
    p.add_argument("--tune-batch", action="store_true",
                   help="with --autotune, also choose the node batch (4k-64k) among those that keep every "
                        "tuning scan's best score")
    p.add_argument("--host-driven", action="store_true",
                   help="iterate searches from the host instead of the device-driven graph loop")
    p.add_argument("--no-kernel-timing", action="store_true",
                   help="skip the kernel-timed pass (the roofline's event times): for runs under a profiler, "
                        "which serializes the pass's timing gate")
    return p.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(torch, ws, total_ms, e2e_ms, probes, e2e_probes, device):
    """Whole-job figures of a replicas-only run: the slowest rank's times
    (max) and every rank's probes (sum); identity on one rank."""
    vals = torch.tensor([total_ms, e2e_ms, probes, e2e_probes], dtype=torch.float64, device=device)
    if ws > 1:
        mx = vals[:2].clone()
        sm = vals[2:].clone()
        torch.distributed.all_reduce(mx, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(sm, op=torch.distributed.ReduceOp.SUM)
        vals = torch.cat([mx, sm])
    return tuple(vals.tolist())


def rank_scans(rank: int, n: int) -> list:
    """Scan indices of one rank: each rank localizes its own n scans (replicas
    only, no data exchange)."""
    return [rank * n + i for i in range(n)]


def _workload_desc(w, m_points, k_mean, scans, batch=None):
    scene = ("indoor multi-room floor 100x60x10 m" if w.name == "indoor" else "outdoor city 800x800x40 m")
    beams = 16 if w.name == "indoor" else 64
    return {"workload": f"{scene}, {m_points / 1e6:.2f} M map points, "
                        f"r={w.r} m, {w.levels} levels; {beams}-beam scans of ~{k_mean:.0f} points",
            "form": "plain (one scan per bbs_localize)", "batch": batch or w.batch, "score_frac": w.score_frac,
            "roll_pitch_range_deg": 6.0, "yaw_range": "0..2pi", "distinct_scans": scans,
            "l2": "flushed between timed steps (512 MiB write)"}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def _oracle_sample(w, m, scan, n_nodes, seed, om=None):
    import numpy as np

    import oracle
    om = om or oracle.Maps(m, w.r, w.levels)
    rg = oracle.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(scan), rg)
    rng = np.random.default_rng(seed)
    # nodes spread over every level, translations inside the search window,
    # the mix a search visits (Eq. (11) against each level's map)
    (a0, a1, a2), (b0, b1, b2) = g.wrange()
    nodes = []
    for _ in range(n_nodes):
        l = int(rng.integers(0, w.levels))
        sh = w.levels - 1 - l
        nodes.append([int(rng.integers(a0 << sh, ((b0 + 1) << sh))), int(rng.integers(a1 << sh, ((b1 + 1) << sh))),
                      int(rng.integers(a2 << sh, ((b2 + 1) << sh))),
                      *(int(rng.integers(0, g.N(l)[i])) for i in range(3)), l])
    return om, g, np.array(nodes, np.int32)


def _cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_legs(w, m, scans, n_poses=5):
    """The CPU oracle on the same workload: its map build, its Eq. (11)
    scoring rate on one thread (a bounded random node sample), and its whole
    BnB per planted pose for n_poses scans on all host cores (the OpenMP
    build: Table I's CPU multi-thread configuration (h); the same searches as
    the single-threaded oracle, pinned)."""
    import oracle
    t = time.perf_counter()
    om = oracle.Maps(m, w.r, w.levels)
    build_s = time.perf_counter() - t
    rate, n, dt = cpu_probe_rate(w, m, scans[0], om=om)
    out = {"value": rate, "unit": "probes/s", "cores": 1, "kind": "oracle",
           "sample": f"{n} random nodes over all levels x {len(scans[0])}-point scan, Eq. (11) scoring "
                     f"({dt:.1f} s, single-threaded C oracle on the host)",
           "nproc": os.cpu_count(), "cpu_model": _cpu_model(), "map_build_ms": build_s * 1e3}
    try:
        threads = oracle.threads(os.cpu_count() or 1)
    except ImportError as ex:
        out["bnb_per_pose"] = {"unavailable": str(ex)}
        return out
    rg = oracle.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    ms, probes, found = [], 0, 0
    for s_ in scans[:n_poses]:
        t = time.perf_counter()
        r = oracle.localize(om, s_, rg, score_frac=w.score_frac, batch=w.batch, mt=True)
        ms.append((time.perf_counter() - t) * 1e3)
        probes += r.probes
        found += r.status == oracle.OK
    out["bnb_per_pose"] = {"kind": "oracle, OpenMP build (Table I configuration (h))", "threads": threads,
                           "poses": len(ms), "ms_per_scan": statistics.mean(ms), "ms_per_scan_each": ms,
                           "probes_per_s": probes / (sum(ms) / 1e3), "found": f"{found}/{len(ms)}"}
    return out


def cpu_probe_rate(w, m, scan, target_s=12.0, om=None):
    """Oracle Eq. (11) scoring throughput (probes/s) on one host thread."""
    om, g, nodes = _oracle_sample(w, m, scan, 200, 1, om)
    t = time.perf_counter()
    om.score_nodes(g, scan, nodes)
    dt = time.perf_counter() - t
    n = int(max(200, 200 * target_s / max(dt, 1e-6)))
    om, g, nodes = _oracle_sample(w, m, scan, n, 1, om)
    t = time.perf_counter()
    om.score_nodes(g, scan, nodes[:n])
    dt = time.perf_counter() - t
    return n * len(scan) / dt, n, dt


def run_reference(a):
    """The reference arm: the CPU oracle on the same workload as the GPU arm.
    Each step is one whole BnB (Algorithm 2's canonical iteration) of the
    next of the same --scans planted-pose scans, run by the oracle's OpenMP
    build on every host core (Table I's CPU multi-thread configuration (h);
    the same search as the single-threaded oracle, pinned); probes/s over the
    timed steps.  Without OpenMP it falls back to the single-threaded oracle
    scoring a bounded random node sample per step."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle

    from paper_2310_10023_gb300 import synth
    w = synth.WORKLOADS[a.workload]
    m = synth.make_map(w.scene)
    scans = [synth.make_scan(w.scene, i)[0] for i in rank_scans(0, a.scans)]
    om = oracle.Maps(m, w.r, w.levels)
    rg = oracle.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    try:
        threads = oracle.threads(os.cpu_count() or 1)
        mt = True
    except ImportError:
        threads, mt = 1, False
    times, probes = [], 0
    if mt:
        for i in range(a.warmup + a.steps):
            t = time.perf_counter()
            r = oracle.localize(om, scans[i % a.scans], rg, score_frac=w.score_frac, batch=w.batch, mt=True)
            dt = time.perf_counter() - t
            if i >= a.warmup:
                times.append(dt)
                probes += r.probes
        sample = (f"whole BnB of each step's scan ({a.scans} planted-pose scans cycled, the GPU arm's), "
                  f"OpenMP build of the C oracle on {threads} threads")
    else:
        _, g, nodes = _oracle_sample(w, m, scans[0], 1000, 7, om)
        t = time.perf_counter()
        om.score_nodes(g, scans[0], nodes[:100])
        per_node = (time.perf_counter() - t) / 100
        n = max(50, int(2.0 / max(per_node, 1e-9)))        # ~2 s of oracle work per step
        _, g, nodes = _oracle_sample(w, m, scans[0], n, 7, om)
        for i in range(a.warmup + a.steps):
            t = time.perf_counter()
            om.score_nodes(g, scans[0], nodes)
            if i >= a.warmup:
                times.append(time.perf_counter() - t)
                probes += n * len(scans[0])
        sample = (f"{n} random nodes over all levels x {len(scans[0])}-point scan per step "
                  "(Eq. (11) scoring, single-threaded C oracle; no OpenMP build)")
    total = sum(times)
    v = probes / total
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "probes/s", "n_gpus": ws, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": total / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _workload_desc(w, len(m), statistics.mean(len(s_) for s_ in scans), a.scans),
            "cpu_baseline": {"value": v, "unit": "probes/s", "cores": threads, "kind": "oracle", "sample": sample,
                             "cpu_model": _cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": v, "unit": "probes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_batched(nv, torch, maps, w, stream, n=64, seed=4):
    """64 indoor scans (K log-uniform in [2k, 30k]) localized in one
    bbs_localize_many call vs the same scans one bbs_localize at a time."""
    from paper_2310_10023_gb300 import synth
    ks = synth.loguniform_sizes(seed, n, 2000, 30000)
    scans = [torch.from_numpy(synth.make_scan(w.scene, 500 + i, k=int(k))[0]).cuda() for i, k in enumerate(ks)]
    a = nv.workload_args(w, stream=stream.cuda_stream)
    nv.bbs_localize_many(maps, scans[:8], a.ranges, a.opts)
    for s_ in scans[:4]:
        nv.bbs_localize(maps, s_, a.ranges, a.opts)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    many = nv.bbs_localize_many(maps, scans, a.ranges, a.opts)
    e1.record(stream)
    e1.synchronize()
    t_many = e0.elapsed_time(e1)
    e0.record(stream)
    plain = [nv.bbs_localize(maps, s_, a.ranges, a.opts) for s_ in scans]
    e1.record(stream)
    e1.synchronize()
    t_plain = e0.elapsed_time(e1)
    pm = sum(r.probes for r in many)
    same = sum((r.best_score, list(r.node)) == (q.best_score, list(q.node)) for r, q in zip(many, plain))
    return {"workload": f"{n} indoor scans, K log-uniform 2k-30k (mean {statistics.mean(int(k) for k in ks):.0f})",
            "probes_per_s": pm / (t_many / 1e3), "plain_probes_per_s": pm / (t_plain / 1e3),
            "speedup_vs_plain": t_plain / t_many, "wall_ms": t_many, "plain_wall_ms": t_plain,
            "ms_to_optimum_mean": statistics.mean(r.ms_to_optimum for r in many),
            "plain_ms_to_optimum_mean": statistics.mean(r.ms_to_optimum for r in plain),
            "found": sum(r.status == nv.OK for r in many), "results_equal_plain": f"{same}/{n}"}


def run_exact(nv, torch, stream, workload="room", n_scans=4):
    """The exact-bound mode: levels above the leaves widened so that every
    node's score bounds its leaves' under rotation too.  Nodes scored, peak
    frontier, time per scan and best scores vs the approximate (default)
    bound on the same scans.  On the room workload (whose exhaustive search
    is the reference of the oracle pins) and on the indoor one, where the
    widened coarse levels keep most nodes and the frontier grows to ~10^8."""
    from paper_2310_10023_gb300 import synth
    w = synth.WORKLOADS[workload]
    m = synth.make_map(w.scene)
    md = torch.from_numpy(np.array(m)).cuda()
    maps = nv.bbs_build_maps(md, w.r, w.levels)
    scans_d = [torch.from_numpy(synth.make_scan(w.scene, i)[0]).cuda() for i in range(n_scans)]
    a = nv.workload_args(w, stream=stream.cuda_stream)
    e = max(nv.bbs_exact_dilation(maps, s_, a.ranges, a.opts) for s_ in scans_d)
    em = nv.bbs_build_maps(md, w.r, w.levels, nv.exact_bound_flags(e))
    out = {"workload": f"{workload}, r={w.r} m, {w.levels} levels, {n_scans} scans of "
                       f"{statistics.mean(len(s_) for s_ in scans_d):.0f} points", "extra_dilation": e}
    for name, mp in (("approximate", maps), ("exact", em)):
        nv.bbs_localize(mp, scans_d[0], a.ranges, a.opts)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = [nv.bbs_localize(mp, s_, a.ranges, a.opts) for s_ in scans_d]
        e1.record(stream)
        e1.synchronize()
        out[name] = {"ms_per_scan": e0.elapsed_time(e1) / len(scans_d),
                     "nodes_scored_mean": statistics.mean(r.nodes_scored for r in res),
                     "peak_frontier_max": max(r.peak_frontier for r in res),
                     "best_scores": [r.best_score for r in res]}
        if name == "approximate":
            out["bound_check"] = _bound_check([r.as_dict() for r in res])
    out["same_best_score"] = f"{sum(x == y for x, y in zip(out['approximate']['best_scores'], out['exact']['best_scores']))}/{len(scans_d)}"
    # the exact-bound BnB returns the exhaustive optimum (pinned against brute
    # force), so its best score measures the approximate bound's gap
    gaps = [(e - a) / e for a, e in zip(out["approximate"]["best_scores"], out["exact"]["best_scores"]) if e > 0]
    out["gap_to_exhaustive_optimum"] = {"mean": statistics.mean(gaps) if gaps else None,
                                        "scans_short": sum(g > 0 for g in gaps), "scans": len(gaps)}
    return out


def _bound_check(results):
    """Sec. IV-A's check of the approximate rotational bound over a set of
    searches: children scored while branching, the fraction scoring above
    their parent, and their mean excess (child - parent) / child."""
    c = sum(r["children_scored"] for r in results)
    v = sum(r["bound_violations"] for r in results)
    x = sum(r["bound_excess"] for r in results)
    return {"children_scored": c, "violations": v, "rate": v / c if c else None,
            "mean_excess": x / v if v else None,
            "paper": "0.001 % of cases, about 1.5 % average error (Sec. IV-A)"}


def run_host_queue(nv, torch, maps, w, scans_d, stream):
    """The same searches with the frontier on the host (Algorithm 2's own
    layout: host buckets, per-batch copies) vs the device-resident engine,
    and the depth-first order (Table I's DFS strategy) on the host queue."""
    a = nv.workload_args(w, stream=stream.cuda_stream)
    d = nv.workload_args(w, stream=stream.cuda_stream, flags=nv.SEARCH_DFS)
    out = {}
    for name, fn, ar in (("device_frontier", nv.bbs_localize, a), ("host_frontier", nv.bbs_localize_hostqueue, a),
                         ("host_frontier_dfs", nv.bbs_localize_hostqueue, d)):
        fn(maps, scans_d[0], ar.ranges, ar.opts)
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = [fn(maps, s_, ar.ranges, ar.opts) for s_ in scans_d]
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t) * 1e3
        out[name] = {"ms_per_scan": ms / len(scans_d), "probes_per_s": sum(r.probes for r in res) / (ms / 1e3),
                     "iterations_mean": statistics.mean(r.iterations for r in res),
                     "nodes_scored_mean": statistics.mean(r.nodes_scored for r in res),
                     "h2d_bytes_per_scan": statistics.mean(r.h2d_bytes for r in res),
                     "d2h_bytes_per_scan": statistics.mean(r.d2h_bytes for r in res), "keys": [
                         (r.best_score, tuple(r.node), r.nodes_scored) for r in res]}
    dev, host, dfs = (out[k].pop("keys") for k in ("device_frontier", "host_frontier", "host_frontier_dfs"))
    out["results_equal"] = f"{sum(x == y for x, y in zip(dev, host))}/{len(scans_d)}"
    out["dfs_same_best_score"] = f"{sum(x[0] == y[0] for x, y in zip(dev, dfs))}/{len(scans_d)}"
    out["speedup_device_vs_host"] = out["host_frontier"]["ms_per_scan"] / out["device_frontier"]["ms_per_scan"]
    out["dfs_vs_bfs_nodes"] = out["host_frontier_dfs"]["nodes_scored_mean"] / out["host_frontier"]["nodes_scored_mean"]
    return out


def run_gicp(nv, torch, maps, w, stream, n_scans=8):
    """Local fine registration after the BnB result (Sec. IV): the indoor BnB
    leaf refined by GICP against the map's voxel centroids; time per
    refinement and the translation error to the planted pose before and
    after."""
    import numpy as np
    from paper_2310_10023_gb300 import synth
    m = synth.make_map(w.scene)
    md = torch.from_numpy(np.array(m)).cuda()
    torch.cuda.synchronize()
    t = time.perf_counter()
    target = nv.bbs_gicp_target_build(md, w.r, stream.cuda_stream)
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t) * 1e3
    del md
    a = nv.workload_args(w, stream=stream.cuda_stream)
    go = nv.make_gicp_opts(stream=stream.cuda_stream)
    e0, e1, r0, r1, ms, its, ncorr = [], [], [], [], [], [], []
    for i in range(n_scans):
        s_, pose = synth.make_scan(w.scene, i)
        sd = torch.from_numpy(s_).cuda()
        res = nv.bbs_localize(maps, sd, a.ranges, a.opts)
        if res.status != nv.OK:
            continue
        R0, t0 = nv.bbs_pose_matrix(res.pose)
        nv.bbs_gicp(target, sd, R0, t0, go)   # warm
        torch.cuda.synchronize()
        t = time.perf_counter()
        g = nv.bbs_gicp(target, sd, R0, t0, go)
        torch.cuda.synchronize()
        ms.append((time.perf_counter() - t) * 1e3)
        its.append(g.iterations)
        ncorr.append(g.correspondences / len(s_))
        Rt, tt = nv.bbs_pose_matrix(pose)
        Rg, tg = g.Rt()
        e0.append(float(np.linalg.norm(t0 - tt)))
        e1.append(float(np.linalg.norm(tg - tt)))
        r0.append(float(np.arccos(np.clip((np.trace(R0.T @ Rt) - 1) / 2, -1, 1))))
        r1.append(float(np.arccos(np.clip((np.trace(Rg.T @ Rt) - 1) / 2, -1, 1))))
    info = nv.bbs_gicp_target_info(target)
    return {"workload": f"indoor, BnB leaf of {len(ms)} scans refined against {info['voxels']} voxel centroids "
                        f"(r = {w.r} m) of the {len(m) / 1e6:.1f} M-point map",
            "ms_per_refinement": statistics.mean(ms) if ms else None,
            "iterations_mean": statistics.mean(its) if its else None,
            "correspondence_fraction": statistics.mean(ncorr) if ncorr else None,
            "translation_error_m": {"bnb": statistics.mean(e0) if e0 else None,
                                    "refined": statistics.mean(e1) if e1 else None},
            "rotation_error_rad": {"bnb": statistics.mean(r0) if r0 else None,
                                   "refined": statistics.mean(r1) if r1 else None},
            "target_build_ms": build_ms}


def _form(fn, *args):
    """An optional form: its failure is reported in the line, not raised."""
    try:
        return fn(*args)
    except Exception as ex:   # noqa: BLE001 -- any failure of a side form is a reported result
        return {"error": f"{type(ex).__name__}: {ex}"}


def run_outdoor(nv, torch, stream, nsm=152, gather_gbs=None, n_scans=4, reps=2):
    """The outdoor workload (800 x 800 x 40 m city, 40 M map points, r = 1 m,
    8 levels, 20 k-point scans): plain probes/s and ms per scan, and the
    scoring kernel's roofline from a kernel-timed pass over the same scans."""
    from paper_2310_10023_gb300 import synth
    w = synth.WORKLOADS["outdoor"]
    m = synth.make_map(w.scene)
    md = torch.from_numpy(np.array(m)).cuda()
    torch.cuda.synchronize()
    t = time.perf_counter()
    maps = nv.bbs_build_maps(md, w.r, w.levels)
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t) * 1e3
    del md
    scans = [torch.from_numpy(synth.make_scan(w.scene, i)[0]).cuda() for i in range(n_scans)]
    a = nv.workload_args(w, stream=stream.cuda_stream)
    for s_ in scans[:2]:
        nv.bbs_localize(maps, s_, a.ranges, a.opts)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = []
    e0.record(stream)
    for _ in range(reps):
        res += [nv.bbs_localize(maps, s_, a.ranges, a.opts) for s_ in scans]
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    probes = sum(r.probes for r in res)
    at = nv.workload_args(w, stream=stream.cuda_stream, flags=nv.TIME_KERNELS)
    with Clocks(torch.cuda.current_device()) as clk:
        kres = [nv.bbs_localize(maps, s_, at.ranges, at.opts) for s_ in scans for _ in range(reps)]
    kms = sum(r.score_ms for r in kres)
    kc = clk.summary() or {}
    roof = _roofline(sum(r.gathers for r in kres) / (kms / 1e3) if kms > 0 else 0.0, kms,
                     sum(r.score_launches for r in kres), kc.get("sm_mhz") or 2070.0, nsm, "outdoor", gather_gbs,
                     rot_per_unit=sum(r.rotations for r in kres) / max(1, sum(r.gathers for r in kres)))
    return {"roofline": roof,
            "workload": f"outdoor city 800x800x40 m, {len(m) / 1e6:.1f} M map points, r={w.r} m, {w.levels} levels; "
                        f"{n_scans} scans of ~{statistics.mean(len(s_) for s_ in scans):.0f} points",
            "probes_per_s": probes / (ms / 1e3), "ms_per_scan": ms / len(res),
            "ms_to_optimum_mean": statistics.mean(r.ms_to_optimum for r in res),
            "found": f"{sum(r.status == nv.OK for r in res)}/{len(res)}", "map_build_ms": build_ms}


def _served_maps(nv, torch):
    from paper_2310_10023_gb300 import synth
    maps = {}
    for name in ("room", "indoor"):
        w = synth.WORKLOADS[name]
        maps[name] = (w, nv.bbs_build_maps(torch.from_numpy(np.array(synth.make_map(w.scene))).cuda(), w.r, w.levels))
    return maps


def run_served(nv, torch, maps, lam=200.0, n=64, seed=9, max_active=4):
    """Poisson arrivals (rate lam) of requests with 2k-30k-point scans against
    two resident maps (room and indoor), served by the continuous-batching
    server, vs one-at-a-time plain BnB on the same arrival trace (FIFO: each
    request's service time measured alone, queued in arrival order)."""
    from paper_2310_10023_gb300 import synth
    arr, ks = synth.poisson_trace(seed, lam, n, 2000, 30000)
    reqs = []
    for i in range(n):
        name = "room" if i % 2 == 0 else "indoor"
        w, dm = maps[name]
        s = synth.make_scan(w.scene, 900 + 100 * seed + i, k=int(ks[i]))[0]
        a = nv.workload_args(w, stream=0)
        reqs.append((dm, s, a.ranges, a.opts))
    # one-at-a-time service times (device synchronized per request)
    torch.cuda.synchronize()
    for dm, s, rg, op in reqs[:4]:
        nv.bbs_localize(dm, s, rg, op)
    svc = []
    for dm, s, rg, op in reqs:
        t = time.perf_counter()
        nv.bbs_localize(dm, s, rg, op)
        svc.append((time.perf_counter() - t) * 1e3)
    fifo, free_at = [], 0.0
    for t_arr, d in zip(arr * 1e3, svc):
        start = max(t_arr, free_at)
        free_at = start + d
        fifo.append(free_at - t_arr)
    srv = nv.bbs_server_create(max_active=max_active)
    tickets = []
    t0 = time.perf_counter()
    for (dm, s, rg, op), t_arr in zip(reqs, arr):
        while time.perf_counter() - t0 < t_arr:
            pass
        tickets.append(nv.bbs_server_submit(srv, dm, s, rg, op))
    out = [nv.bbs_server_poll(srv, t, -1) for t in tickets]
    st = nv.bbs_server_stats(srv)
    srv.close()
    q = sorted(fifo)
    pct = lambda v, p: v[min(len(v) - 1, int(round(p * (len(v) - 1))))]
    return {"rate_rps": lam, "requests": n, "max_active": max_active, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "throughput_rps": st["throughput_rps"], "probes_per_s": st["probes_per_s"],
            "peak_active": st["peak_active"], "found": sum(o[0] == nv.OK for o in out),
            "plain_fifo_p50_ms": pct(q, 0.5), "plain_fifo_p99_ms": pct(q, 0.99),
            "plain_throughput_rps": n / (max(free_at, arr[-1] * 1e3) / 1e3),
            "plain_mean_service_ms": statistics.mean(svc)}


def run_served_sweep(nv, torch, rates=(20, 50, 100, 200, 500, 1000), n=128, max_active=4):
    """The served form over arrival rates from light load to overload (one
    seeded trace per rate), each against one-at-a-time FIFO on its trace.
    At most max_active requests share the device loop: each shared launch
    lengthens every member's iterations, and beyond a few members the
    throughput gained is small while every request's latency keeps growing."""
    maps = _served_maps(nv, torch)
    out = {"workload": f"{n} requests per rate, Poisson arrivals, K log-uniform 2k-30k, maps room + indoor "
                       f"resident, at most {max_active} requests in the device loop at once; plain: one "
                       "bbs_localize at a time in arrival order (FIFO)",
           "rates": [run_served(nv, torch, maps, float(lam), n, seed=9 + j, max_active=max_active)
                     for j, lam in enumerate(rates)]}
    return out


def _kernel_hash():
    """Hash of the scoring kernel's source files with their comments and
    blank lines removed (a comment edit keeps a capture valid)."""
    h = hashlib.sha256()
    for f in ("branch.cu", "bbs_internal.cuh", "branch.cuh"):
        src = open(os.path.join(ROOT, "paper_2310_10023_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in src.splitlines()]
        h.update("\n".join(ln for ln in lines if ln.strip()).encode())
    return h.hexdigest()[:16]


def _profile_kv(workload=WORKLOAD):
    """The machine-readable lines ("- key: `value`") of the committed ncu
    summary of the scoring kernel on a workload
    (profiles/branch3_kernel_<workload>.md), if it was taken on the current
    kernel source; else {}."""
    p = os.path.join(ROOT, "profiles", f"branch3_kernel_{workload}.md")
    if not os.path.exists(p):
        return {}
    kv = {}
    for line in open(p):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("kernel_hash") != _kernel_hash():
        return {}
    out = {}
    for k, v in kv.items():
        try:
            out[k] = float(v)
        except ValueError:
            out[k] = v
    return out


def _by_launch_size(log, peak_gops, ops_per_unit):
    """The scoring launches split at their median size: units, device time and
    the ALU fraction of the smaller and the larger half (ops per unit: the
    run's average, the launch log holds units only)."""
    if not log:
        return None
    log = sorted(log)
    half = len(log) // 2
    out = {}
    for name, part in (("smaller_half", log[:half]), ("larger_half", log[half:])):
        u = sum(x for x, _ in part)
        t = sum(y for _, y in part)
        out[name] = {"launches": len(part), "units_mean": u / len(part) if part else None, "ms": t,
                     "frac": (u / (t / 1e3) * ops_per_unit / 1e9) / peak_gops if t > 0 else None}
    return out


def _roofline(units_per_s, score_ms, launches, sm_mhz, nsm, workload, gather_peak_gbs=None, rot_per_unit=1.0):
    """The scoring kernel's roofline.  Bound: ALU issue (L1 serves most of its
    probes).  Algorithmic work: OPS_PER_PROBE per unit (one scan point x one
    rotational child, which answers its 8 translational children) plus
    OPS_PER_ROTATION per rotated scan point, counted as the kernel rotates
    them (once per run of tasks that share a rotation: rot_per_unit rotated
    points per unit); peak: SMs x 128 INT32/FP32 lanes x the SM clock sampled
    during the timed region.  The L2 and L1 sector rates come from the
    committed ncu capture of the same kernel source (sectors and duration of
    the captured launches), the L2 peak from this run's random-gather
    plateau."""
    alu_peak = nsm * 128 * sm_mhz * 1e6 / 1e9          # Gop/s
    ops_per_unit = OPS_PER_PROBE + OPS_PER_ROTATION * rot_per_unit
    achieved = units_per_s * ops_per_unit / 1e9
    kv = _profile_kv(workload)
    out = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Gop/s", "frac": achieved / alu_peak,
           "traffic": kv.get("dram_bytes_per_launch"),
           "kernel": "branch3_kernel (fused branch + Eq. (11) scoring)",
           "algorithmic_ops": f"{OPS_PER_PROBE} per scan point per rotational child (3 translation adds, 8 child "
                              f"counts) + {OPS_PER_ROTATION} per rotated scan point (9 products, 6 sums, 3 floors); "
                              f"{rot_per_unit:.4f} rotated points per unit here: {ops_per_unit:.2f} per unit",
           "units_per_s": units_per_s, "rotated_points_per_unit": rot_per_unit, "launches": launches,
           "kernel_ms": score_ms,
           "peak_source": f"{nsm} SMs x 128 lanes x {sm_mhz:.0f} MHz (median SM clock in the timed region)"}
    dur = kv.get("duration_us_per_launch")
    if dur:
        l2 = kv.get("lts_sectors_per_launch", 0.0) * 32 / (dur * 1e-6) / 1e9
        l1 = kv.get("l1_sectors_per_launch", 0.0) * 32 / (dur * 1e-6) / 1e9
        out["l2"] = {"achieved": l2, "peak": gather_peak_gbs, "unit": "GB/s",
                     "frac": l2 / gather_peak_gbs if gather_peak_gbs else None,
                     "source": f"lts__t_sectors / gpu__time_duration of profiles/branch3_kernel_{workload}.md; "
                               "peak: random 32-byte gathers over an L2-resident table (bbs_bench_gather, this run)"}
        out["l1"] = {"achieved": l1, "unit": "GB/s",
                     "source": "l1tex__t_sectors_pipe_lsu_mem_global_op_ld / gpu__time_duration, same capture"}
    return out


def run_ours(a):
    import numpy as np
    import torch

    from paper_2310_10023_gb300 import build, native as nv, synth

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if not os.path.exists(nv.LIB_PATH):
        build.build()
    nv.load()
    stream = torch.cuda.current_stream()

    w = synth.WORKLOADS[a.workload]
    m = synth.make_map(w.scene)
    md = torch.from_numpy(np.array(m)).to(dev)
    scans = [synth.make_scan(w.scene, i)[0] for i in rank_scans(rank, a.scans)]
    scans_d = [torch.from_numpy(s).to(dev) for s in scans]
    tuning = None
    batch = w.batch
    if a.autotune or a.tune_batch:
        from paper_2310_10023_gb300 import autotune
        props = torch.cuda.get_device_properties(dev)
        targs = nv.workload_args(w, stream=stream.cuda_stream)
        out = autotune.tuned(props.name, props.multi_processor_count, lambda: nv.bbs_build_maps(md, w.r, w.levels),
                             scans_d[:4], targs.ranges, targs.opts, w.r, w.levels, [len(s) for s in scans],
                             tune_batch=a.tune_batch)
        tuning = dict(out["best"], cached=out["cached"])
        if a.tune_batch:
            batch = int(out["batch"])
            tuning["batch"] = batch
    torch.cuda.synchronize()
    t = time.perf_counter()
    maps = nv.bbs_build_maps(md, w.r, w.levels)
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t) * 1e3
    del md
    args = nv.workload_args(w, stream=stream.cuda_stream, flags=nv.TIME_KERNELS, batch=batch)
    args_plain = nv.workload_args(w, stream=stream.cuda_stream, batch=batch,
                                  flags=nv.HOST_DRIVEN if a.host_driven else 0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up (both the device-driven path and the kernel-timed path)
    for i in range(a.warmup):
        nv.bbs_localize(maps, scans_d[i % a.scans], args_plain.ranges, args_plain.opts)
        if not a.no_kernel_timing:
            nv.bbs_localize(maps, scans_d[i % a.scans], args.ranges, args.opts)

    # ---- timed: device-resident scans (device-driven search loop) -------------
    launch_log = []   # (units, ms) of every scoring launch of the kernel-timed steps

    def timed_steps(opts):
        res, ms = [], []
        barrier()
        with Clocks(torch.cuda.current_device()) as clk:
            for i in range(a.steps):
                flush.zero_()
                # the call's host work must not overlap the flush: the GPU is
                # idle when the timed region starts
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = nv.bbs_localize(maps, scans_d[i % a.scans], args.ranges, opts)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
                res.append(r.as_dict())
                if opts.flags & nv.TIME_KERNELS:
                    launch_log.extend(zip(*nv.bbs_launch_log()))
        barrier()
        return res, ms, clk.summary()

    results, step_ms, clocks = timed_steps(args_plain.opts)
    total_ms = sum(step_ms)
    probes = sum(r["probes"] for r in results)
    launches = sum(r["launches"] for r in results)
    to_opt = statistics.mean(r["ms_to_optimum"] for r in results)
    # where one scan's time goes (the library's own per-result phases, medians)
    phase_names = ("setup", "initial_enqueue", "device_to_match", "device_after_match", "readback")
    phases = {n: statistics.median(r["phase_ms"][j] for r in results) for j, n in enumerate(phase_names)}
    found = sum(r["status"] == nv.OK for r in results)
    # ---- timed again with every scoring launch bracketed by CUDA events on the
    # stream (host-driven iterations: the graph's loop body cannot hold events)
    kres, kclocks = [], None
    if not a.no_kernel_timing:
        kres, _, kclocks = timed_steps(args.opts)
    score_ms = sum(r["score_ms"] for r in kres)
    score_launches = sum(r["score_launches"] for r in kres)
    gathers = sum(r["gathers"] for r in kres)
    rotations = sum(r["rotations"] for r in kres)

    # ---- timed: host buffers through the same C-ABI call ------------------
    e2e_ms = []
    h2d = d2h = 0
    barrier()
    for i in range(a.steps):
        flush.zero_()
        torch.cuda.synchronize()
        s = scans[i % a.scans]
        t = time.perf_counter()
        r = nv.bbs_localize(maps, s, args_plain.ranges, args_plain.opts)
        e2e_ms.append((time.perf_counter() - t) * 1e3)
        h2d += r.h2d_bytes          # scan, angle tables, control block: counted by the library
        d2h += r.d2h_bytes          # per-iteration control block and the result
    barrier()
    e2e_total = sum(e2e_ms)
    e2e_probes = probes  # the same scans in the same order

    # ---- rooflines (measured live) -------------------------------------------
    units_per_s = gathers / (score_ms / 1e3) if score_ms > 0 else 0.0
    sm_mhz = (kclocks or clocks or {}).get("sm_mhz") or 2070.0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    # the L2 random-gather plateau over a table of the level-0 table's size
    lvl0 = nv.bbs_maps_info(maps, 0)
    table_bytes = lvl0["table_size"] * (1 if lvl0["layout"] == nv.LAYOUT_BYTES else 32)
    gb = 1 << 27
    peak_ms = min(nv.bbs_bench_gather(max(table_bytes, 1 << 22), gb, stream.cuda_stream) for _ in range(3))
    gather_gbs = gb * 32 / peak_ms / 1e6
    roofline = _roofline(units_per_s, score_ms, score_launches, sm_mhz, nsm, a.workload, gather_gbs,
                         rot_per_unit=rotations / gathers if gathers else 1.0)
    roofline["by_launch_size"] = _by_launch_size(launch_log, roofline["peak"],
                                                 OPS_PER_PROBE + OPS_PER_ROTATION * roofline["rotated_points_per_unit"])

    # ---- reduce over ranks ----------------------------------------------------
    total_ms, e2e_total, probes_all, e2e_probes_all = reduce_over_ranks(torch, ws, total_ms, e2e_total, probes,
                                                                        e2e_probes, dev)

    batched = served = exact = outdoor = host_queue = refine = None
    if rank == 0 and ws == 1 and not a.no_forms:
        batched = _form(run_batched, nv, torch, maps, w, stream)
        served = _form(run_served_sweep, nv, torch)
        exact = {"room": _form(run_exact, nv, torch, stream, "room", 4),
                 "indoor": _form(run_exact, nv, torch, stream, "indoor", 2)}
        outdoor = _form(run_outdoor, nv, torch, stream, nsm, gather_gbs)
        host_queue = _form(run_host_queue, nv, torch, maps, w, scans_d, stream)
        refine = _form(run_gicp, nv, torch, maps, w, stream)
    cpu = None
    if rank == 0 and ws == 1 and not a.no_cpu_baseline:
        cpu = cpu_legs(w, m, scans)
    if rank == 0:
        line = {
            "metric": METRIC, "value": probes_all / (total_ms / 1e3), "unit": "probes/s", "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(_workload_desc(w, len(m), statistics.mean(len(s) for s in scans), a.scans, batch),
                           launch_shape=tuning or dict(nv.bbs_get_tuning(), layout=0, load_factor=0.25, source="defaults"),
                           map_layout=sorted({nv.LAYOUT_NAMES[nv.bbs_maps_layout(maps, l)] for l in range(w.levels)})),
            "ms_to_optimum": to_opt,
            "ms_total_per_scan": total_ms / a.steps,
            "ms_per_scan_median": statistics.median(step_ms),
            "phase_ms_median": dict(phases, note="setup: scan upload, d_max, pose grid, angle tables, slot; "
                                                 "initial_enqueue: host time to launch the initial set; "
                                                 "device_*: %globaltimer from the initial set's start"),
            "found": f"{found}/{a.steps}",
            "map_build_ms": build_ms,
            "bound_check": _bound_check(results),
            "roofline": roofline,
            "batched": batched,
            "served": served,
            "exact_bound": exact,
            "outdoor": outdoor,
            "host_queue": host_queue,
            "gicp": refine,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_probes_all / (e2e_total / 1e3), "unit": "probes/s",
                    "h2d_bytes_per_step": h2d // a.steps, "d2h_bytes_per_step": d2h // a.steps},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()

"""ctypes binding of libbbs (include/bbs.h): same names, argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays
and torch tensors to pointers, picks host or device residency from the
arguments, and turns status codes into exceptions.  Loading fails loudly when
libbbs.so has not been built -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbbs.so")

OK, NOT_FOUND, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EKEYRANGE, ECORRUPT = 0, 1, -1, -2, -3, -4, -5, -6
ECANCELED, PENDING = -7, 2
TRANSLATION_ONLY, LEAF_UNDILATED, PRUNE_GE, ANGLE_LOWER_EDGE, CHILD_LITERAL = 0x1, 0x2, 0x4, 0x8, 0x10
SEARCH_DFS = 0x40          # depth-first batched order (bbs_localize_hostqueue)
TIME_KERNELS, HOST_DRIVEN = 0x100, 0x200
EXACT_BOUND = 0x20


def exact_bound_flags(e: int) -> int:
    """bbs_build_maps flags of the exact-bound mode with extra dilation e (1..15)."""
    return EXACT_BOUND | (int(e) << 12)
MAX_LEVELS = 16

_lock = threading.Lock()
_lib = None


class BBSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libbbs error {code}: {msg}")
        self.code = code


class Ranges(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("ang_lo", C.c_double * 3), ("ang_hi", C.c_double * 3)]


class Opts(C.Structure):
    _fields_ = [("score_frac", C.c_double), ("batch", C.c_int64), ("d_max", C.c_double),
                ("flags", C.c_uint32), ("cuda_stream", C.c_void_p), ("max_frontier", C.c_int64)]


class Result(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("found", C.c_int32), ("best_score", C.c_int32), ("num_points", C.c_int32),
        ("node", C.c_int32 * 7), ("pose", C.c_double * 6),
        ("nodes_scored", C.c_int64), ("probes", C.c_int64), ("iterations", C.c_int64),
        ("peak_frontier", C.c_int64), ("parents_branched", C.c_int64),
        ("ms_to_optimum", C.c_double), ("ms_total", C.c_double), ("phase_ms", C.c_double * 5),
        ("gathers", C.c_int64), ("launches", C.c_int64), ("score_launches", C.c_int64), ("score_ms", C.c_double),
        ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64),
        ("children_scored", C.c_int64), ("bound_violations", C.c_int64), ("bound_excess", C.c_double),
        ("rotations", C.c_int64),
    ]

    def as_dict(self) -> dict:
        return {
            "status": self.status, "found": self.found, "best_score": self.best_score,
            "num_points": self.num_points, "node": list(self.node), "pose": list(self.pose),
            "nodes_scored": self.nodes_scored, "probes": self.probes, "iterations": self.iterations,
            "peak_frontier": self.peak_frontier, "parents_branched": self.parents_branched,
            "ms_to_optimum": self.ms_to_optimum, "ms_total": self.ms_total, "phase_ms": list(self.phase_ms),
            "gathers": self.gathers, "launches": self.launches, "score_launches": self.score_launches,
            "score_ms": self.score_ms, "h2d_bytes": self.h2d_bytes, "d2h_bytes": self.d2h_bytes,
            "children_scored": self.children_scored, "bound_violations": self.bound_violations,
            "bound_excess": self.bound_excess, "rotations": self.rotations,
        }


class GicpOpts(C.Structure):
    """bbs_gicp_opts (0 = default)."""
    _fields_ = [("max_iters", C.c_int32), ("pad", C.c_int32), ("tau", C.c_double), ("rho", C.c_double),
                ("cov_eps", C.c_double), ("eps_rot", C.c_double), ("eps_trans", C.c_double),
                ("cuda_stream", C.c_void_p)]


class GicpResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("converged", C.c_int32), ("iterations", C.c_int32),
                ("correspondences", C.c_int32), ("cost", C.c_double), ("R", C.c_double * 9), ("t", C.c_double * 3),
                ("pose", C.c_double * 6), ("ms", C.c_double)]

    def Rt(self):
        return np.array(list(self.R)).reshape(3, 3), np.array(list(self.t))


class Tuning(C.Structure):
    """bbs_tuning: launch shape of the search (0 = default)."""
    _fields_ = [("launch_tasks", C.c_int64), ("static_pm", C.c_int32), ("grab_min", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("frontier_log2", C.c_int32)]

    def as_dict(self):
        return {"launch_tasks": self.launch_tasks, "static_pm": self.static_pm, "grab_min": self.grab_min,
                "ctas_per_sm": self.ctas_per_sm, "frontier_log2": self.frontier_log2}


class ServerOpts(C.Structure):
    _fields_ = [("mem_budget", C.c_size_t), ("max_active", C.c_int32), ("max_frontier", C.c_int64)]


class ServerCounters(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("active", C.c_int64), ("queued", C.c_int64),
                ("rejected", C.c_int64), ("peak_active", C.c_int64), ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_ms", C.c_double),
                ("throughput_rps", C.c_double), ("probes_per_s", C.c_double), ("mem_in_use", C.c_size_t),
                ("mem_budget", C.c_size_t)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ("bbs_build_maps", "bbs_free_maps", "bbs_maps_bbox", "bbs_maps_info", "bbs_maps_keys",
           "bbs_pose_grid", "bbs_score_batch", "bbs_score_children", "bbs_localize", "bbs_last_error",
           "bbs_version")


def load():
    """Load libbbs.so; raise if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2310_10023_gb300.build.build() "
                              "(the CUDA library is required; there is no fallback)")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER
        vp, i64, i32p, f32p, i64p, dp = C.c_void_p, C.c_int64, P(C.c_int32), C.c_void_p, P(C.c_int64), P(C.c_double)
        L.bbs_build_maps.argtypes = [vp, i64, C.c_int, C.c_float, C.c_int, C.c_uint32, vp, P(C.c_void_p)]
        L.bbs_free_maps.argtypes = [vp]
        L.bbs_free_maps.restype = None
        L.bbs_maps_bbox.argtypes = [vp, dp, dp]
        L.bbs_maps_info.argtypes = [vp, C.c_int, i64p, i64p, i64p, i32p, dp]
        L.bbs_maps_keys.argtypes = [vp, C.c_int, vp, i64, i64p]
        L.bbs_maps_layout.argtypes = [vp, C.c_int, i32p]
        L.bbs_maps_device.argtypes = [vp, i32p]
        L.bbs_pose_matrix.argtypes = [vp, vp, vp]
        L.bbs_gicp_target_build.argtypes = [vp, i64, C.c_int, C.c_float, vp, P(C.c_void_p)]
        L.bbs_gicp_target_free.argtypes = [vp]
        L.bbs_gicp_target_free.restype = None
        L.bbs_gicp_target_info.argtypes = [vp, i64p, i64p, i32p]
        L.bbs_gicp.argtypes = [vp, vp, i64, C.c_int, vp, vp, P(GicpOpts), P(GicpResult)]
        L.bbs_gicp_linearize.argtypes = [vp, vp, i64, C.c_int, vp, vp, P(GicpOpts), vp, vp, P(C.c_double), i64p, vp, vp]
        L.bbs_pose_grid.argtypes = [vp, vp, i64, C.c_int, P(Ranges), P(Opts), C.c_int, i64p, vp, i64, i64p]
        L.bbs_score_batch.argtypes = [vp, vp, i64, C.c_int, P(Ranges), P(Opts), vp, i64, vp]
        L.bbs_score_children.argtypes = [vp, vp, i64, C.c_int, P(Ranges), P(Opts), vp, i64, vp, vp, i64, i64p]
        L.bbs_localize.argtypes = [vp, vp, i64, C.c_int, P(Ranges), P(Opts), P(Result)]
        L.bbs_localize_many.argtypes = [vp, C.c_int, P(C.c_void_p), P(C.c_int64), C.c_int, P(Ranges), P(Opts),
                                        P(Result)]
        L.bbs_last_error.restype = C.c_char_p
        L.bbs_version.restype = C.c_char_p
        L.bbs_set_load_factor.argtypes = [C.c_double]
        L.bbs_set_probe_layout.argtypes = [C.c_int]
        L.bbs_set_tuning.argtypes = [C.c_void_p]
        L.bbs_localize_hostqueue.argtypes = [vp, vp, i64, C.c_int, vp, vp, vp]
        L.bbs_exact_dilation.argtypes = [vp, vp, i64, C.c_int, vp, vp, i32p]
        L.bbs_get_tuning.argtypes = [C.c_void_p]
        L.bbs_launch_log.argtypes = [vp, vp, i64, i64p]
        L.bbs_server_create.argtypes = [P(ServerOpts), P(C.c_void_p)]
        L.bbs_server_submit.argtypes = [vp, vp, vp, i64, P(Ranges), P(Opts), P(C.c_uint64)]
        L.bbs_server_poll.argtypes = [vp, C.c_uint64, C.c_int, P(Result)]
        L.bbs_server_cancel.argtypes = [vp, C.c_uint64]
        L.bbs_server_stats.argtypes = [vp, P(ServerCounters)]
        L.bbs_server_destroy.argtypes = [vp]
        L.bbs_server_destroy.restype = None
        L.bbs_bench_gather.argtypes = [C.c_int64, C.c_int64, vp, P(C.c_double)]
        L.bbs_score_batch_noalloc.argtypes = [vp, vp, i64, P(Ranges), P(Opts), vp, i64, vp]
        _lib = L
        return L


def bbs_last_error() -> str:
    return load().bbs_last_error().decode()


def bbs_version() -> str:
    return load().bbs_version().decode()


def _check(rc: int, allow_not_found=False) -> int:
    if rc == OK or (allow_not_found and rc == NOT_FOUND):
        return rc
    raise BBSError(rc, bbs_last_error())


# ---- argument marshalling --------------------------------------------------

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _arr(x, dtype, cols=None):
    """-> (pointer, is_device, n_rows, keepalive)."""
    if _is_torch(x):
        import torch
        tdt = {np.float32: torch.float32, np.int32: torch.int32}[dtype]
        t = x.detach()
        if t.dtype != tdt:
            raise TypeError(f"expected {tdt}, got {t.dtype}")
        t = t.contiguous()
        n = t.shape[0] if t.dim() > 0 else 0
        if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
            raise ValueError(f"expected shape (n, {cols}), got {tuple(t.shape)}")
        return C.c_void_p(t.data_ptr()), 1 if t.is_cuda else 0, n, t
    a = np.ascontiguousarray(x, dtype=dtype)
    if cols is not None:
        a = a.reshape(-1, cols)
    return C.c_void_p(a.ctypes.data), 0, a.shape[0], a


def make_ranges(lo, hi, ang_lo, ang_hi) -> Ranges:
    r = Ranges()
    for i in range(3):
        r.lo[i], r.hi[i] = float(lo[i]), float(hi[i])
        r.ang_lo[i], r.ang_hi[i] = float(ang_lo[i]), float(ang_hi[i])
    return r


def make_opts(score_frac=0.0, batch=0, d_max=0.0, flags=0, stream=None, max_frontier=0) -> Opts:
    o = Opts()
    o.score_frac = float(score_frac)
    o.batch = int(batch)
    o.d_max = float(d_max)
    o.flags = int(flags)
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                stream = torch.cuda.current_stream().cuda_stream
        except Exception:  # noqa: BLE001 - torch is optional here
            stream = None
    o.cuda_stream = C.c_void_p(int(stream) if stream else 0)
    o.max_frontier = int(max_frontier)
    return o


class Maps:
    """Owning handle of a device-resident voxel-map pyramid."""

    def __init__(self, handle: C.c_void_p, r: float, levels: int, flags: int):
        self.h = handle
        self.r = r
        self.levels = levels
        self.flags = flags

    def close(self):
        if getattr(self, "h", None):
            load().bbs_free_maps(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


# ---- the C-ABI, one function each -------------------------------------------

def bbs_build_maps(xyz, r: float, levels: int, flags: int = 0, stream=None) -> Maps:
    p, dev, n, keep = _arr(xyz, np.float32, 3)
    h = C.c_void_p()
    st = make_opts(stream=stream).cuda_stream
    _check(load().bbs_build_maps(p, n, dev, C.c_float(r), int(levels), int(flags), st, C.byref(h)))
    del keep
    return Maps(h, float(np.float32(r)), int(levels), int(flags))


def bbs_free_maps(maps: Maps) -> None:
    maps.close()


def bbs_maps_bbox(maps: Maps):
    lo, hi = (C.c_double * 3)(), (C.c_double * 3)()
    _check(load().bbs_maps_bbox(maps.h, lo, hi))
    return tuple(lo), tuple(hi)


def bbs_maps_info(maps: Maps, level: int) -> dict:
    nv, nb, ts = C.c_int64(), C.c_int64(), C.c_int64()
    mp, cr = C.c_int32(), C.c_double()
    _check(load().bbs_maps_info(maps.h, int(level), C.byref(nv), C.byref(nb), C.byref(ts), C.byref(mp), C.byref(cr)))
    return {"voxels": nv.value, "buckets": nb.value, "table_size": ts.value, "max_probe": mp.value,
            "collision_rate": cr.value, "layout": bbs_maps_layout(maps, level)}


LAYOUT_WIDE, LAYOUT_COMPACT, LAYOUT_DENSE, LAYOUT_BYTES = 0, 1, 2, 3
LAYOUT_NAMES = {LAYOUT_WIDE: "wide", LAYOUT_COMPACT: "compact", LAYOUT_DENSE: "dense", LAYOUT_BYTES: "bytes"}


def bbs_maps_layout(maps: Maps, level: int) -> int:
    """Table layout of one level: LAYOUT_WIDE, LAYOUT_COMPACT, LAYOUT_DENSE or LAYOUT_BYTES."""
    out = C.c_int32()
    _check(load().bbs_maps_layout(maps.h, int(level), C.byref(out)))
    return out.value


def bbs_maps_device(maps: Maps) -> int:
    """The CUDA device index holding the maps."""
    out = C.c_int32()
    _check(load().bbs_maps_device(maps.h, C.byref(out)))
    return out.value


def bbs_maps_keys(maps: Maps, level: int) -> np.ndarray:
    n = bbs_maps_info(maps, level)["voxels"]
    out = np.zeros((max(n, 1), 3), np.int32)
    got = C.c_int64()
    _check(load().bbs_maps_keys(maps.h, int(level), C.c_void_p(out.ctypes.data), n, C.byref(got)))
    return out[:got.value]


def bbs_pose_grid(maps: Maps, scan, ranges: Ranges | None = None, opts: Opts | None = None, level: int = 0,
                  tables: bool = True):
    """-> (dims dict, (n_rot, 9) float32 rotation table or None)."""
    p, dev, k, keep = _arr(scan, np.float32, 3)
    opts = opts or make_opts()
    dims = (C.c_int64 * 12)()
    nrot = C.c_int64()
    _check(load().bbs_pose_grid(maps.h, p, k, dev, C.byref(ranges) if ranges else None, C.byref(opts), int(level),
                                dims, None, 0, C.byref(nrot)))
    A = None
    if tables:
        A = np.zeros((nrot.value, 9), np.float32)
        _check(load().bbs_pose_grid(maps.h, p, k, dev, C.byref(ranges) if ranges else None, C.byref(opts),
                                    int(level), dims, C.c_void_p(A.ctypes.data), nrot.value, C.byref(nrot)))
    del keep
    d = list(dims)
    return {"N": tuple(d[0:3]), "a": tuple(d[3:6]), "wmin": tuple(d[6:9]), "wmax": tuple(d[9:12]),
            "n_rot": nrot.value}, A


def bbs_score_batch(maps: Maps, scan, nodes, ranges: Ranges | None = None, opts: Opts | None = None, out=None):
    """Eq. (11) scores of caller nodes (n x 7 int32).  Device tensors in, device tensor out."""
    sp, sdev, k, keep1 = _arr(scan, np.float32, 3)
    npt, ndev, n, keep2 = _arr(nodes, np.int32, 7)
    if sdev != ndev:
        raise ValueError("scan and nodes must both be host or both be device memory")
    if out is None:
        if ndev:
            import torch
            out = torch.empty(n, dtype=torch.int32, device=keep2.device)
        else:
            out = np.zeros(n, np.int32)
    op, odev, _, keep3 = _arr(out, np.int32)
    if odev != ndev:
        raise ValueError("scores must have the residency of nodes")
    opts = opts or make_opts()
    _check(load().bbs_score_batch(maps.h, sp, k, sdev, C.byref(ranges) if ranges else None, C.byref(opts),
                                  npt, n, op))
    del keep1, keep2
    return keep3 if keep3 is not out and not _is_torch(out) else out


NOALLOC_MAX_POINTS = 131072
NOALLOC_MAX_ANGLES = 65536


def bbs_score_batch_noalloc(maps: Maps, scan, nodes, scores, ranges: Ranges | None = None,
                            opts: Opts | None = None):
    """Scores of caller nodes into the caller's `scores`, with no allocation
    inside the library: scan, nodes and scores must be device tensors on the
    maps' device, and scores contiguous (it is written in place).  For callers
    that cannot allocate while they run (real-time loops, external memory
    pools).  The library's scratch array is shared by every call."""
    if not all(_is_torch(x) for x in (scan, nodes, scores)):
        raise ValueError("bbs_score_batch_noalloc takes device tensors only")
    dev = bbs_maps_device(maps)
    for name, x in (("scan", scan), ("nodes", nodes), ("scores", scores)):
        if not x.is_cuda or x.device.index != dev:
            raise ValueError(f"{name} must be on cuda:{dev}, the maps' device (got {x.device})")
    if not scores.is_contiguous():
        raise ValueError("scores must be contiguous: it is written in place")
    sp, sdev, k, keep1 = _arr(scan, np.float32, 3)
    npt, ndev, n, keep2 = _arr(nodes, np.int32, 7)
    op, odev, no, keep3 = _arr(scores, np.int32)
    if no < n:
        raise ValueError("scores is shorter than nodes")
    opts = opts or make_opts()
    _check(load().bbs_score_batch_noalloc(maps.h, sp, k, C.byref(ranges) if ranges else None, C.byref(opts),
                                          npt, n, op))
    del keep1, keep2, keep3
    return scores


def bbs_score_children(maps: Maps, scan, parents, ranges: Ranges | None = None, opts: Opts | None = None):
    """Children (Eq. (13)) of each parent with their scores, canonical order."""
    sp, sdev, k, keep1 = _arr(scan, np.float32, 3)
    pp, pdev, n, keep2 = _arr(parents, np.int32, 7)
    if sdev or pdev:
        raise ValueError("bbs_score_children binding takes host arrays")
    opts = opts or make_opts()
    cnt = C.c_int64()
    rg = C.byref(ranges) if ranges else None
    rc = load().bbs_score_children(maps.h, sp, k, 0, rg, C.byref(opts), pp, n, None, None, 0, C.byref(cnt))
    if rc not in (OK, EINVAL) or (rc == EINVAL and cnt.value == 0 and n > 0):
        _check(rc)
    nodes = np.zeros((max(cnt.value, 1), 7), np.int32)
    scores = np.zeros(max(cnt.value, 1), np.int32)
    _check(load().bbs_score_children(maps.h, sp, k, 0, rg, C.byref(opts), pp, n, C.c_void_p(nodes.ctypes.data),
                                     C.c_void_p(scores.ctypes.data), cnt.value, C.byref(cnt)))
    del keep1, keep2
    return nodes[:cnt.value], scores[:cnt.value]


def bbs_localize(maps: Maps, scan, ranges: Ranges | None = None, opts: Opts | None = None) -> Result:
    p, dev, k, keep = _arr(scan, np.float32, 3)
    opts = opts or make_opts()
    res = Result()
    _check(load().bbs_localize(maps.h, p, k, dev, C.byref(ranges) if ranges else None, C.byref(opts),
                               C.byref(res)), allow_not_found=True)
    del keep
    return res


def bbs_localize_hostqueue(maps: Maps, scan, ranges: Ranges | None = None, opts: Opts | None = None) -> Result:
    """bbs_localize with the frontier on the host (Algorithm 2's own layout):
    same results, per-batch copies to and from the GPU."""
    p, dev, k, keep = _arr(scan, np.float32, 3)
    opts = opts or make_opts()
    res = Result()
    _check(load().bbs_localize_hostqueue(maps.h, p, k, dev, C.byref(ranges) if ranges else None, C.byref(opts),
                                         C.byref(res)), allow_not_found=True)
    del keep
    return res


class GicpTarget:
    """Owned bbs_gicp_target handle (freed on garbage collection)."""

    def __init__(self, h):
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.bbs_gicp_target_free(self.h)
            self.h = None


def bbs_gicp_target_build(xyz, r: float, stream=None) -> GicpTarget:
    """The GICP target of a map cloud: its points grouped by fine voxel key (centroids)."""
    p, dev, n, keep = _arr(xyz, np.float32, 3)
    h = C.c_void_p()
    _check(load().bbs_gicp_target_build(p, n, dev, float(r), C.c_void_p(stream) if stream else None, C.byref(h)))
    del keep
    return GicpTarget(h)


def bbs_gicp_target_free(t: GicpTarget) -> None:
    """Free a target now (otherwise it is freed with the handle object)."""
    if t.h:
        load().bbs_gicp_target_free(t.h)
        t.h = None


def bbs_gicp_target_info(t: GicpTarget) -> dict:
    nv_, ts, mp = C.c_int64(), C.c_int64(), C.c_int32()
    _check(load().bbs_gicp_target_info(t.h, C.byref(nv_), C.byref(ts), C.byref(mp)))
    return {"voxels": nv_.value, "table_size": ts.value, "max_probe": mp.value}


def bbs_pose_matrix(pose):
    """(x, y, z, roll, pitch, yaw) -> (R 3x3, t 3) in FP64: the library's pose
    convention (the transform of bbs_result.pose and bbs_gicp's seed)."""
    p = np.ascontiguousarray([float(v) for v in pose], np.float64)
    if p.shape != (6,):
        raise ValueError("a pose has 6 entries")
    R = np.zeros(9)
    t = np.zeros(3)
    _check(load().bbs_pose_matrix(C.c_void_p(p.ctypes.data), C.c_void_p(R.ctypes.data), C.c_void_p(t.ctypes.data)))
    return R.reshape(3, 3), t


def make_gicp_opts(max_iters=0, tau=0.0, rho=0.0, cov_eps=0.0, eps_rot=0.0, eps_trans=0.0, stream=None) -> GicpOpts:
    o = GicpOpts()
    o.max_iters, o.tau, o.rho, o.cov_eps = int(max_iters), float(tau), float(rho), float(cov_eps)
    o.eps_rot, o.eps_trans = float(eps_rot), float(eps_trans)
    o.cuda_stream = C.c_void_p(stream) if stream else None
    return o


def bbs_gicp(target: GicpTarget, scan, R0, t0, opts: GicpOpts | None = None) -> GicpResult:
    """GICP refinement of a scan's pose (R0, t0) against a target's voxel centroids."""
    p, dev, k, keep = _arr(scan, np.float32, 3)
    R = np.ascontiguousarray(R0, np.float64).reshape(9)
    t = np.ascontiguousarray(t0, np.float64).reshape(3)
    res = GicpResult()
    _check(load().bbs_gicp(target.h, p, k, dev, C.c_void_p(R.ctypes.data), C.c_void_p(t.ctypes.data),
                           C.byref(opts or make_gicp_opts()), C.byref(res)))
    del keep
    return res


def bbs_gicp_linearize(target: GicpTarget, scan, R, t, opts: GicpOpts | None = None, per_point: bool = True):
    """One linearization at (R, t) -> (H 6x6, g 6, cost, n, voxels (k, 3), found (k,))."""
    p, dev, k, keep = _arr(scan, np.float32, 3)
    Ra = np.ascontiguousarray(R, np.float64).reshape(9)
    ta = np.ascontiguousarray(t, np.float64).reshape(3)
    H = np.zeros(36)
    g = np.zeros(6)
    cost = C.c_double()
    n = C.c_int64()
    vox = np.zeros((max(k, 1), 3), np.int32)
    found = np.zeros(max(k, 1), np.uint8)
    _check(load().bbs_gicp_linearize(target.h, p, k, dev, C.c_void_p(Ra.ctypes.data), C.c_void_p(ta.ctypes.data),
                                     C.byref(opts or make_gicp_opts()), C.c_void_p(H.ctypes.data),
                                     C.c_void_p(g.ctypes.data), C.byref(cost), C.byref(n),
                                     C.c_void_p(vox.ctypes.data) if per_point else None,
                                     C.c_void_p(found.ctypes.data) if per_point else None))
    del keep
    return H.reshape(6, 6), g, cost.value, n.value, vox[:k], found[:k].astype(bool)


def bbs_localize_many(maps: Maps, scans, ranges: Ranges | None = None, opts: Opts | None = None) -> list:
    """Localize several scans (list of (K_i, 3) arrays / tensors, all host or all
    device) in shared launches; one Result per scan."""
    n = len(scans)
    ptrs = (C.c_void_p * max(n, 1))()
    ks = (C.c_int64 * max(n, 1))()
    keep = []
    dev = None
    for i, sc in enumerate(scans):
        p, d, k, kp = _arr(sc, np.float32, 3)
        if dev is None:
            dev = d
        elif d != dev:
            raise ValueError("scans must all be host or all be device memory")
        ptrs[i] = p.value
        ks[i] = k
        keep.append(kp)
    opts = opts or make_opts()
    res = (Result * max(n, 1))()
    _check(load().bbs_localize_many(maps.h, n, ptrs, ks, int(dev or 0), C.byref(ranges) if ranges else None,
                                    C.byref(opts), res))
    del keep
    return [res[i] for i in range(n)]


class Server:
    """Owning handle of a continuous-batching server (bbs_server_*)."""

    def __init__(self, h):
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().bbs_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def bbs_server_create(mem_budget: int = 0, max_active: int = 0, max_frontier: int = 0) -> Server:
    o = ServerOpts(int(mem_budget), int(max_active), int(max_frontier))
    h = C.c_void_p()
    _check(load().bbs_server_create(C.byref(o), C.byref(h)))
    return Server(h)


def bbs_server_submit(server: Server, maps: Maps, scan, ranges: Ranges | None = None,
                      opts: Opts | None = None) -> int:
    p, dev, k, keep = _arr(scan, np.float32, 3)
    if dev:
        raise ValueError("bbs_server_submit takes a host scan (it is copied)")
    t = C.c_uint64()
    _check(load().bbs_server_submit(server.h, maps.h, p, k, C.byref(ranges) if ranges else None,
                                    C.byref(opts or make_opts(stream=0)), C.byref(t)))
    del keep
    return t.value


def bbs_server_poll(server: Server, ticket: int, wait_ms: int = -1):
    """-> (status, Result or None); status PENDING while queued or running."""
    res = Result()
    rc = load().bbs_server_poll(server.h, int(ticket), int(wait_ms), C.byref(res))
    if rc == PENDING:
        return rc, None
    if rc == EINVAL and res.status == 0 and res.num_points == 0:
        _check(rc)
    return rc, res


def bbs_server_cancel(server: Server, ticket: int) -> None:
    _check(load().bbs_server_cancel(server.h, int(ticket)))


def bbs_server_stats(server: Server) -> dict:
    c = ServerCounters()
    _check(load().bbs_server_stats(server.h, C.byref(c)))
    return c.as_dict()


def bbs_server_destroy(server: Server) -> None:
    server.close()


def bbs_exact_dilation(maps: Maps, scan, ranges=None, opts=None) -> int:
    """Extra dilation the exact-bound mode needs for this scan (-1: none can)."""
    p, dev, n, keep = _arr(scan, np.float32, 3)
    e = C.c_int32()
    _check(load().bbs_exact_dilation(maps.h, p, n, dev, C.byref(ranges) if ranges is not None else None,
                                     C.byref(opts) if opts is not None else None, C.byref(e)))
    del keep
    return int(e.value)


def bbs_set_tuning(launch_tasks: int = 0, static_pm: int = 0, grab_min: int = 0, ctas_per_sm: int = 0,
                   frontier_log2: int = 0, reset: bool = False) -> None:
    """Launch shape of later searches (0 = default); reset=True restores every default."""
    if reset:
        _check(load().bbs_set_tuning(None))
        return
    t = Tuning(int(launch_tasks), int(static_pm), int(grab_min), int(ctas_per_sm), int(frontier_log2))
    _check(load().bbs_set_tuning(C.byref(t)))


def bbs_launch_log():
    """(units, ms) of each scoring launch of the last BBS_TIME_KERNELS search
    call on this thread: numpy arrays (rotational children x scan points per
    launch, device milliseconds)."""
    n = C.c_int64()
    rc = load().bbs_launch_log(None, None, 0, C.byref(n))
    units = np.zeros(max(n.value, 1), np.int64)
    ms = np.zeros(max(n.value, 1), np.float64)
    if n.value:
        _check(load().bbs_launch_log(C.c_void_p(units.ctypes.data), C.c_void_p(ms.ctypes.data), n.value, C.byref(n)))
    else:
        _check(rc)
    return units[:n.value], ms[:n.value]


def bbs_get_tuning() -> dict:
    t = Tuning()
    _check(load().bbs_get_tuning(C.byref(t)))
    return t.as_dict()


def bbs_set_load_factor(load_factor: float) -> None:
    _check(load().bbs_set_load_factor(float(load_factor)))


def bbs_set_probe_layout(layout: int) -> None:
    """0 (default): byte grid where a level's box is small enough, else
    compact where it fits, else wide; 1: always wide; 2: hashed only;
    3: dense bricks where the box qualifies; 4: byte grid where it does."""
    _check(load().bbs_set_probe_layout(int(layout)))


def bbs_bench_gather(table_bytes: int, gathers: int, stream=None) -> float:
    """Device milliseconds of `gathers` random 32-byte bucket reads."""
    ms = C.c_double()
    _check(load().bbs_bench_gather(int(table_bytes), int(gathers), make_opts(stream=stream).cuda_stream,
                                   C.byref(ms)))
    return ms.value


@dataclass
class Workload:
    """Convenience bundle of ranges/opts for a synthetic workload."""
    ranges: Ranges
    opts: Opts


def workload_args(w, stream=None, **kw) -> Workload:
    return Workload(make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi),
                    make_opts(score_frac=kw.pop("score_frac", w.score_frac), batch=kw.pop("batch", w.batch),
                              stream=stream, **kw))

"""CPU oracle for 3D-BBS (arxiv 2310.10023) -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``oracle.c`` (plain single-threaded C,
FP64 grid, FP32 keys with no FMA) through ctypes and shares no code with the
CUDA library.  Each wrapper names the passage of the paper it follows:

* ``delta`` -- Sec. III-B, Eq. (2)
* ``Grid`` -- Sec. III-B Eq. (3)-(5), Sec. III-D Eq. (12), (14)
* ``Maps`` -- Sec. III-C, Eq. (10) and the dilation of the last paragraph
* ``Maps.score_nodes`` -- Sec. III-C, Eq. (11)
* ``children`` -- Sec. III-D, Eq. (13)
* ``localize`` -- Sec. III-E, Algorithm 2 (canonical best-first iteration)
* ``brute_force`` -- Sec. III-B, Eq. (1) over the leaf set
* ``threads`` / ``mt=True`` -- the same code built with OpenMP: Table I's CPU
  multi-thread configurations (Sec. IV), scoring loops in parallel
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_LIB_MT_PATH = os.path.join(_HERE, "liborc_mt.so")   # the same source with OpenMP (Table I's CPU multi-thread rows)
_lock = threading.Lock()
_lib = None
_lib_mt = None

OK, NOT_FOUND, EINVAL, ENOMEM, EKEYRANGE = 0, 1, -1, -2, -5
TRANSLATION_ONLY, LEAF_UNDILATED, PRUNE_GE, ANGLE_LOWER_EDGE, CHILD_LITERAL = 0x1, 0x2, 0x4, 0x8, 0x10
EXACT_BOUND = 0x20
SEARCH_DFS = 0x40          # depth-first batched order (localize only)


def exact_flags(e: int) -> int:
    """Map flags of the exact-bound mode with extra dilation e (1..15)."""
    return EXACT_BOUND | (int(e) << 12)
MAX_LEVELS = 16


def _compile(out, extra, force):
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
        os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", *extra, "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile liborc.so with gcc (no FMA contraction, no fast-math), and
    liborc_mt.so, the same source with OpenMP, where gcc supports it."""
    path = _compile(_LIB_PATH, ["-Wno-unknown-pragmas"], force)
    try:
        _compile(_LIB_MT_PATH, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        pass   # no OpenMP here: the multi-thread variant is unavailable
    return path


class Ranges(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("ang_lo", C.c_double * 3), ("ang_hi", C.c_double * 3)]


class GridT(C.Structure):
    _fields_ = [
        ("levels", C.c_int), ("r", C.c_double), ("d_max", C.c_double), ("flags", C.c_uint32),
        ("ang_lo", C.c_double * 3), ("ang_range", C.c_double * 3),
        ("delta", C.c_double * MAX_LEVELS),
        ("N", (C.c_int64 * 3) * MAX_LEVELS),
        ("dprime", (C.c_double * 3) * MAX_LEVELS),
        ("a", (C.c_int64 * 3) * MAX_LEVELS),
        ("wmin", C.c_int64 * 3), ("wmax", C.c_int64 * 3),
    ]


class ResultT(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("found", C.c_int32), ("best_score", C.c_int32), ("num_points", C.c_int32),
        ("node", C.c_int32 * 7), ("pose", C.c_double * 6),
        ("nodes_scored", C.c_int64), ("probes", C.c_int64), ("iterations", C.c_int64),
        ("peak_frontier", C.c_int64), ("parents_branched", C.c_int64), ("ms_total", C.c_double),
        ("children_scored", C.c_int64), ("bound_violations", C.c_int64), ("bound_excess", C.c_double),
    ]


def _load(mt: bool = False):
    """The oracle library; mt=True: its OpenMP build (ImportError when gcc
    had no OpenMP)."""
    global _lib, _lib_mt
    with _lock:
        if (_lib_mt if mt else _lib) is not None:
            return _lib_mt if mt else _lib
        build()
        if mt and not os.path.exists(_LIB_MT_PATH):
            raise ImportError("liborc_mt.so was not built (no OpenMP in this gcc)")
        L = C.CDLL(_LIB_MT_PATH if mt else _LIB_PATH)
        P = C.POINTER
        f32p, i32p, i64p, dp = P(C.c_float), P(C.c_int32), P(C.c_int64), P(C.c_double)
        L.orc_delta.restype = C.c_double
        L.orc_delta.argtypes = [C.c_double, C.c_double]
        L.orc_scan_dmax.restype = C.c_double
        L.orc_scan_dmax.argtypes = [f32p, C.c_int64]
        L.orc_grid_build.argtypes = [C.c_double, C.c_int, C.c_double, P(Ranges), C.c_uint32, P(GridT)]
        L.orc_angle.restype = C.c_double
        L.orc_angle.argtypes = [P(GridT), C.c_int, C.c_int, C.c_int64]
        L.orc_exact_dilation.restype = C.c_int
        L.orc_exact_dilation.argtypes = [P(GridT), C.c_double]
        L.orc_rotation.restype = None
        L.orc_rotation.argtypes = [P(GridT), C.c_int, C.c_int64, C.c_int64, C.c_int64, f32p]
        L.orc_num_children.restype = C.c_int64
        L.orc_num_children.argtypes = [P(GridT), i32p]
        L.orc_children.restype = C.c_int64
        L.orc_children.argtypes = [P(GridT), i32p, i32p, C.c_int64]
        L.orc_maps_build.argtypes = [f32p, C.c_int64, C.c_float, C.c_int, C.c_uint32, P(C.c_void_p)]
        L.orc_maps_free.restype = None
        L.orc_maps_free.argtypes = [C.c_void_p]
        for name in ("orc_maps_count", "orc_maps_table_size", "orc_maps_collisions"):
            getattr(L, name).restype = C.c_int64
            getattr(L, name).argtypes = [C.c_void_p, C.c_int]
        L.orc_maps_keys.restype = C.c_int64
        L.orc_maps_keys.argtypes = [C.c_void_p, C.c_int, i32p, C.c_int64]
        L.orc_maps_contains.argtypes = [C.c_void_p, C.c_int, C.c_int32, C.c_int32, C.c_int32]
        L.orc_maps_bbox.restype = None
        L.orc_maps_bbox.argtypes = [C.c_void_p, dp, dp]
        L.orc_score.restype = C.c_int32
        L.orc_score.argtypes = [C.c_void_p, P(GridT), f32p, C.c_int64, i32p]
        L.orc_score_nodes.argtypes = [C.c_void_p, P(GridT), f32p, C.c_int64, i32p, C.c_int64, i32p]
        L.orc_localize.argtypes = [C.c_void_p, f32p, C.c_int64, P(Ranges), C.c_double, C.c_int64,
                                   C.c_double, C.c_uint32, C.c_int64, P(ResultT)]
        L.orc_brute_force.argtypes = [C.c_void_p, P(GridT), f32p, C.c_int64, i32p, i32p]
        L.orc_threads.argtypes = [C.c_int]
        if mt:
            _lib_mt = L
        else:
            _lib = L
        return L


def threads(n: int = 0) -> int:
    """Threads of the OpenMP oracle (n > 0 sets them): the CPU multi-thread
    configurations of Table I.  The searches and scores are the plain
    oracle's; only the scoring loops run in parallel."""
    return _load(mt=True).orc_threads(int(n))


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(C.POINTER(C.c_float))


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def make_ranges(lo, hi, ang_lo, ang_hi) -> Ranges:
    r = Ranges()
    for i in range(3):
        r.lo[i], r.hi[i] = float(lo[i]), float(hi[i])
        r.ang_lo[i], r.ang_hi[i] = float(ang_lo[i]), float(ang_hi[i])
    return r


def delta(r: float, d_max: float) -> float:
    """Eq. (2) with the argument clamped to [-1, 1]."""
    return _load().orc_delta(float(r), float(d_max))


def scan_dmax(scan) -> float:
    s, p = _f32(scan)
    return _load().orc_scan_dmax(p, len(s))


class Grid:
    """Pose grid of Sec. III-B / III-D for one (map, scan, ranges) triple."""

    def __init__(self, r: float, levels: int, d_max: float, ranges: Ranges, flags: int = 0):
        self.g = GridT()
        rc = _load().orc_grid_build(float(np.float32(r)), int(levels), float(d_max), C.byref(ranges),
                                    int(flags), C.byref(self.g))
        if rc != OK:
            raise ValueError(f"orc_grid_build failed: {rc}")

    @property
    def levels(self):
        return self.g.levels

    def N(self, l):
        return tuple(self.g.N[l][i] for i in range(3))

    def dprime(self, l):
        return tuple(self.g.dprime[l][i] for i in range(3))

    def a(self, l):
        return tuple(self.g.a[l][i] for i in range(3))

    def delta(self, l):
        return self.g.delta[l]

    def wrange(self):
        return tuple(self.g.wmin[i] for i in range(3)), tuple(self.g.wmax[i] for i in range(3))

    def angle(self, l, axis, c):
        return _load().orc_angle(C.byref(self.g), l, axis, int(c))

    def rotation(self, l, ia, ib, ig) -> np.ndarray:
        A = np.zeros(9, np.float32)
        _load().orc_rotation(C.byref(self.g), l, int(ia), int(ib), int(ig),
                             A.ctypes.data_as(C.POINTER(C.c_float)))
        return A

    def rotation_table(self, l) -> np.ndarray:
        na, nb, ng = self.N(l)
        out = np.zeros((na * nb * ng, 9), np.float32)
        i = 0
        for a in range(na):
            for b in range(nb):
                for g in range(ng):
                    out[i] = self.rotation(l, a, b, g)
                    i += 1
        return out

    def num_children(self, node) -> int:
        n, p = _i32(node)
        return _load().orc_num_children(C.byref(self.g), p)

    def exact_dilation(self, scan_norm_max: float = 0.0) -> int:
        """Extra dilation the exact-bound mode needs for this grid (-1: none can)."""
        return _load().orc_exact_dilation(C.byref(self.g), float(scan_norm_max))

    def children(self, node) -> np.ndarray:
        n, p = _i32(node)
        cnt = _load().orc_children(C.byref(self.g), p, None, 0)
        out = np.zeros((max(cnt, 1), 7), np.int32)
        _load().orc_children(C.byref(self.g), p, out.ctypes.data_as(C.POINTER(C.c_int32)), cnt)
        return out[:cnt]


class Maps:
    """Per-level sparse hash voxel maps with dilation (Sec. III-C)."""

    def __init__(self, xyz, r: float, levels: int, flags: int = 0):
        x, p = _f32(xyz)
        h = C.c_void_p()
        rc = _load().orc_maps_build(p, len(x), float(r), int(levels), int(flags), C.byref(h))
        self.status = rc
        if rc != OK:
            raise ValueError(f"orc_maps_build failed: {rc}")
        self.h = h
        self.r = float(np.float32(r))
        self.levels = levels
        self.flags = flags

    def __del__(self):
        if getattr(self, "h", None):
            _load().orc_maps_free(self.h)
            self.h = None

    def count(self, l):
        return _load().orc_maps_count(self.h, l)

    def table_size(self, l):
        return _load().orc_maps_table_size(self.h, l)

    def collisions(self, l):
        return _load().orc_maps_collisions(self.h, l)

    def keys(self, l) -> np.ndarray:
        n = self.count(l)
        out = np.zeros((max(n, 1), 3), np.int32)
        _load().orc_maps_keys(self.h, l, out.ctypes.data_as(C.POINTER(C.c_int32)), n)
        return out[:n]

    def contains(self, l, v) -> bool:
        return bool(_load().orc_maps_contains(self.h, l, int(v[0]), int(v[1]), int(v[2])))

    def bbox(self):
        lo = (C.c_double * 3)()
        hi = (C.c_double * 3)()
        _load().orc_maps_bbox(self.h, lo, hi)
        return tuple(lo), tuple(hi)

    def score_nodes(self, grid: Grid, scan, nodes, mt: bool = False) -> np.ndarray:
        s, sp = _f32(scan)
        n, np_ = _i32(np.asarray(nodes).reshape(-1, 7))
        out = np.zeros(len(n), np.int32)
        rc = _load(mt).orc_score_nodes(self.h, C.byref(grid.g), sp, len(s), np_, len(n),
                                       out.ctypes.data_as(C.POINTER(C.c_int32)))
        if rc != OK:
            raise ValueError(f"orc_score_nodes failed: {rc}")
        return out


def localize(maps: Maps, scan, ranges: Ranges, score_frac=0.95, batch=10000, d_max=0.0, flags=0,
             max_frontier=0, mt: bool = False) -> ResultT:
    """Canonical best-first batched BnB (Algorithm 2 with the reading in
    oracle.c); mt=True runs the OpenMP build (same result, scoring loops in
    parallel)."""
    s, sp = _f32(scan)
    res = ResultT()
    _load(mt).orc_localize(maps.h, sp, len(s), C.byref(ranges), float(score_frac), int(batch),
                           float(d_max), int(flags), int(max_frontier), C.byref(res))
    return res


def brute_force(maps: Maps, grid: Grid, scan):
    """Exhaustive maximum of Eq. (11) over every leaf of the grid."""
    s, sp = _f32(scan)
    best = C.c_int32()
    node = (C.c_int32 * 7)()
    rc = _load().orc_brute_force(maps.h, C.byref(grid.g), sp, len(s), C.byref(best), node)
    if rc != OK:
        raise ValueError(f"orc_brute_force failed: {rc}")
    return int(best.value), tuple(node)

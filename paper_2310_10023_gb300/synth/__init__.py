"""Seeded synthetic workloads for 3D-BBS: maps, scans, search ranges, traces.

Inputs only -- this module holds none of the localization arithmetic.  The
scenes stand in for the paper's simulated urban and real outdoor datasets,
which are not available: a 20 x 20 x 5 m room (r = 0.5 m, 3 levels), a
100 x 60 x 10 m multi-room floor (~5 M points, r = 0.2 m, 6 levels) and an
800 x 800 x 40 m city block grid (~40 M points, r = 1.0 m, 8 levels).
"""
from __future__ import annotations

import ctypes as C
import functools
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libbbs_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "synth.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall",
                    "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            P = C.POINTER
            L.syn_map.argtypes = [C.c_int, C.c_int64, P(P(C.c_float)), P(C.c_int64)]
            L.syn_scan.argtypes = [C.c_int, C.c_int, C.c_int64, P(P(C.c_float)), P(C.c_int64),
                                   P(C.c_double)]
            L.syn_free.argtypes = [C.c_void_p]
            L.syn_free.restype = None
            L.syn_scene_extent.argtypes = [C.c_int, P(C.c_double), P(C.c_double)]
            L.syn_trace.argtypes = [C.c_uint64, C.c_double, C.c_int64, C.c_int64, C.c_int64,
                                    P(C.c_double), P(C.c_int64)]
            L.syn_trace.restype = None
            L.syn_mt64.argtypes = [C.c_uint64, C.c_int64, P(C.c_uint64)]
            L.syn_mt64.restype = None
            _lib = L
    return _lib


def _take(ptr, n) -> np.ndarray:
    arr = np.ctypeslib.as_array(ptr, shape=(n * 3,)).copy().reshape(n, 3) if n > 0 else np.zeros((0, 3), np.float32)
    _load().syn_free(ptr)
    return arr


@functools.lru_cache(maxsize=4)
def _map_cached(cfg: int, n_override: int) -> np.ndarray:
    p = C.POINTER(C.c_float)()
    n = C.c_int64()
    if _load().syn_map(cfg, n_override, C.byref(p), C.byref(n)) != 0:
        raise ValueError(f"unknown scene {cfg}")
    a = _take(p, n.value)
    a.setflags(write=False)
    return a


def make_map(scene: int, n_points: int = 0) -> np.ndarray:
    """(N, 3) float32 map cloud of scene 1 (room), 2 (indoor floor) or 3 (city)."""
    return _map_cached(int(scene), int(n_points))


def make_scan(scene: int, index: int, k: int = 0):
    """Scan `index` of a scene -> ((K, 3) float32 sensor-frame points, planted
    pose (x, y, z, roll, pitch, yaw)).  k > 0 asks for exactly k points."""
    p = C.POINTER(C.c_float)()
    n = C.c_int64()
    pose = (C.c_double * 6)()
    if _load().syn_scan(int(scene), int(index), int(k), C.byref(p), C.byref(n), pose) != 0:
        raise ValueError(f"unknown scene {scene}")
    return _take(p, n.value), tuple(pose)


def scene_extent(scene: int):
    lo = (C.c_double * 3)()
    hi = (C.c_double * 3)()
    _load().syn_scene_extent(int(scene), lo, hi)
    return tuple(lo), tuple(hi)


def poisson_trace(seed: int, lam: float, n: int, kmin: int = 2000, kmax: int = 30000):
    """Arrival times (s) and scan sizes (log-uniform) of a Poisson request trace."""
    arr = np.zeros(n, np.float64)
    ks = np.zeros(n, np.int64)
    _load().syn_trace(seed, lam, n, kmin, kmax, arr.ctypes.data_as(C.POINTER(C.c_double)),
                      ks.ctypes.data_as(C.POINTER(C.c_int64)))
    return arr, ks


def loguniform_sizes(seed: int, n: int, kmin: int = 2000, kmax: int = 30000) -> np.ndarray:
    _, ks = poisson_trace(seed, 1.0, n, kmin, kmax)
    return ks


def mt64(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, np.uint64)
    _load().syn_mt64(seed, n, out.ctypes.data_as(C.POINTER(C.c_uint64)))
    return out


DEG = math.pi / 180.0


@dataclass(frozen=True)
class Workload:
    """One workload: scene, voxel size r, levels L and search ranges."""
    name: str
    scene: int
    r: float
    levels: int
    lo: tuple
    hi: tuple
    ang_lo: tuple = (-3 * DEG, -3 * DEG, 0.0)
    ang_hi: tuple = (3 * DEG, 3 * DEG, 2 * math.pi)
    score_frac: float = 0.95
    batch: int = 10000


WORKLOADS = {
    # 20 x 20 x 5 m room, r = 0.5 m, 3 levels, full-room translation
    "room": Workload("room", 1, 0.5, 3, (0.0, 0.0, 0.0), (20.0, 20.0, 5.0)),
    # 100 x 60 x 10 m indoor floor, r = 0.2 m, 6 levels
    "indoor": Workload("indoor", 2, 0.2, 6, (0.0, 0.0, 0.0), (100.0, 60.0, 10.0), batch=16384),
    # 800 x 800 x 40 m city, r = 1 m, 8 levels, 400 x 400 x 10 m window
    "outdoor": Workload("outdoor", 3, 1.0, 8, (200.0, 200.0, -3.0), (600.0, 600.0, 7.0), batch=16384),
}

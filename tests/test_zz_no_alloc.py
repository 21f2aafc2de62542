"""bbs_score_batch_noalloc: the scores of bbs_score_batch without any allocation
inside the library, for callers that cannot allocate while they run (real-time
loops that must not touch an allocator after start-up, frameworks owning all
device memory).  Checked against the CPU oracle's Eq. (11) scores and against
the allocating entry point, exactly (integer scores), on two calls in a row so
that the shared scratch array's leftovers from the first call cannot leak into
the second; and checked to allocate nothing: the device's default memory pool
(cudaMallocAsync) keeps its high-water mark and reservation, and the device's
free memory (cudaMalloc) is unchanged across the two calls.  Collected last on
purpose."""
import ctypes

import numpy as np
import pytest

from paper_2310_10023_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# CUmemPool_attribute values of the driver API (cuda.h)
_RESERVED_MEM_CURRENT, _USED_MEM_CURRENT, _USED_MEM_HIGH = 5, 7, 8


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_10023_gb300 import build, native
    build.build()
    native.load()
    return native


class _Memory:
    """The device's default memory pool and free memory, through the driver API."""

    def __init__(self, device):
        try:
            self.cu = ctypes.CDLL("libcuda.so.1")
        except OSError:
            pytest.skip("libcuda.so.1 not loadable")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), int(device)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def attr(self, a):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, a, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = ctypes.c_uint64(0)      # resets the high-water mark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, _USED_MEM_HIGH, ctypes.byref(z)) == 0

    def free(self):
        f, t = ctypes.c_size_t(), ctypes.c_size_t()
        assert self.cu.cuMemGetInfo_v2(ctypes.byref(f), ctypes.byref(t)) == 0
        return f.value


def _nodes(rng, n, levels, N_of_level):
    out = []
    for _ in range(n):
        l = int(rng.integers(0, levels))
        out.append([int(rng.integers(-2, (42 >> l) + 1)), int(rng.integers(-2, (42 >> l) + 1)),
                    int(rng.integers(-1, (11 >> l) + 1)), *(int(rng.integers(0, N_of_level(l)[i])) for i in range(3)), l])
    return np.array(out, np.int32)


def test_noalloc_equals_oracle_and_score_batch_twice_without_allocating(nv):
    import oracle
    w = synth.WORKLOADS["room"]
    m = synth.make_map(w.scene)
    maps = nv.bbs_build_maps(m, w.r, w.levels)
    om = oracle.Maps(m, w.r, w.levels)
    rg = nv.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    orng = oracle.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    calls = []
    for call, (scan_index, k) in enumerate([(0, 1000), (4, 613)]):     # a ragged second scan
        s, _ = synth.make_scan(w.scene, scan_index)
        s = np.ascontiguousarray(s[:k])
        g = oracle.Grid(w.r, w.levels, oracle.scan_dmax(s), orng)
        nodes = _nodes(np.random.default_rng(call), 2500, w.levels, g.N)
        want = om.score_nodes(g, s, nodes)
        assert np.array_equal(nv.bbs_score_batch(maps, s, nodes, rg), want), call
        sd, nd = torch.from_numpy(s).cuda(), torch.from_numpy(nodes).cuda()
        out = torch.full((len(nodes),), -7, dtype=torch.int32, device="cuda")
        calls.append((sd, nd, out, want))
    # the first call on the device looks up the scratch array's address
    sd, nd, out, _ = calls[0]
    nv.bbs_score_batch_noalloc(maps, sd, nd, out, rg)
    torch.cuda.synchronize()
    mem = _Memory(torch.cuda.current_device())
    used0, reserved0 = mem.attr(_USED_MEM_CURRENT), mem.attr(_RESERVED_MEM_CURRENT)
    mem.reset_high()
    free0 = mem.free()
    for sd, nd, out, _ in calls:
        out.fill_(-7)
    torch.cuda.synchronize()
    for sd, nd, out, _ in calls:
        nv.bbs_score_batch_noalloc(maps, sd, nd, out, rg)
    torch.cuda.synchronize()
    assert mem.attr(_USED_MEM_HIGH) == used0
    assert mem.attr(_RESERVED_MEM_CURRENT) == reserved0
    assert mem.free() == free0
    for call, (sd, nd, out, want) in enumerate(calls):
        assert np.array_equal(out.cpu().numpy(), want), call


def test_noalloc_rejects_oversize_scan(nv):
    w = synth.WORKLOADS["room"]
    maps = nv.bbs_build_maps(synth.make_map(w.scene), w.r, w.levels)
    big = torch.zeros((nv.NOALLOC_MAX_POINTS + 1, 3), dtype=torch.float32, device="cuda")
    nodes = torch.zeros((1, 7), dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(nv.BBSError) as e:
        nv.bbs_score_batch_noalloc(maps, big, nodes, out)
    assert e.value.code == nv.EINVAL
    assert "maximum" in str(e.value)


def test_noalloc_refuses_host_memory_and_strided_scores(nv):
    """Host buffers are refused by the library itself (the pointer check) and
    by the binding; a strided scores tensor would be written to a copy, so
    the binding refuses it."""
    w = synth.WORKLOADS["room"]
    maps = nv.bbs_build_maps(synth.make_map(w.scene), w.r, w.levels)
    s = torch.from_numpy(np.ascontiguousarray(synth.make_scan(w.scene, 0)[0][:100])).cuda()
    nodes = torch.zeros((4, 7), dtype=torch.int32, device="cuda")
    out = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        nv.bbs_score_batch_noalloc(maps, s, nodes, out[::2])
    with pytest.raises(ValueError):
        nv.bbs_score_batch_noalloc(maps, s.cpu(), nodes, out[:4])
    # straight through the C ABI with a host scan pointer
    host = np.ascontiguousarray(s.cpu().numpy())
    opts = nv.make_opts()
    rc = nv.load().bbs_score_batch_noalloc(maps.h, ctypes.c_void_p(host.ctypes.data), len(host), None,
                                           ctypes.byref(opts), ctypes.c_void_p(nodes.data_ptr()), 4,
                                           ctypes.c_void_p(out.data_ptr()))
    assert rc == nv.EINVAL
    assert "device memory" in nv.bbs_last_error()

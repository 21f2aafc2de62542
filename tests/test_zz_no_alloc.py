"""bbs_score_batch_noalloc: the scores of bbs_score_batch without any allocation
inside the library, for callers that cannot allocate while they run (real-time
loops, frameworks owning all device memory).  Compared with the allocating
entry point on the same inputs, exactly (integer scores), on two calls in a row
so that the shared scratch array's leftovers from the first call cannot leak
into the second.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2310_10023_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def nv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_10023_gb300 import build, native
    build.build()
    native.load()
    return native


def _nodes(rng, n, levels, N_of_level):
    out = []
    for _ in range(n):
        l = int(rng.integers(0, levels))
        out.append([int(rng.integers(-2, (42 >> l) + 1)), int(rng.integers(-2, (42 >> l) + 1)),
                    int(rng.integers(-1, (11 >> l) + 1)), *(int(rng.integers(0, N_of_level(l)[i])) for i in range(3)), l])
    return np.array(out, np.int32)


def test_noalloc_equals_score_batch_twice(nv):
    w = synth.WORKLOADS["room"]
    m = synth.make_map(w.scene)
    maps = nv.bbs_build_maps(m, w.r, w.levels)
    rg = nv.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi)
    for call, (scan_index, k) in enumerate([(0, 1000), (4, 613)]):     # a ragged second scan
        s, _ = synth.make_scan(w.scene, scan_index)
        s = np.ascontiguousarray(s[:k])
        dims = [nv.bbs_pose_grid(maps, s, rg, level=l, tables=False)[0]["N"] for l in range(w.levels)]
        nodes = _nodes(np.random.default_rng(call), 2500, w.levels, lambda l: dims[l])
        want = nv.bbs_score_batch(maps, s, nodes, rg)
        sd, nd = torch.from_numpy(s).cuda(), torch.from_numpy(nodes).cuda()
        out = torch.full((len(nodes),), -7, dtype=torch.int32, device="cuda")
        nv.bbs_score_batch_noalloc(maps, sd, nd, out, rg)
        torch.cuda.synchronize()
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

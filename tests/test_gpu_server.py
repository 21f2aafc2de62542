"""The continuous-batching server: requests against two resident maps arrive
while others run, share launches, and each result equals the same request
localized alone and the CPU oracle's search of it; admission follows the
device-memory budget."""
import time

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


@pytest.fixture(scope="module")
def two_maps(nv):
    out = {}
    for name in ("room", "indoor"):
        w = synth.WORKLOADS[name]
        m = synth.make_map(w.scene)
        out[name] = (w, nv.bbs_build_maps(m, w.r, w.levels))
    return out


def _args(nv, w):
    return nv.make_ranges(w.lo, w.hi, w.ang_lo, w.ang_hi), nv.make_opts(score_frac=w.score_frac, batch=w.batch,
                                                                       stream=0)


def _same(a, b):
    return (a.status, a.best_score, list(a.node), a.iterations, a.nodes_scored) == \
           (b.status, b.best_score, list(b.node), b.iterations, b.nodes_scored)


def test_served_results_equal_alone(nv, two_maps):
    srv = nv.bbs_server_create(max_active=8, max_frontier=1 << 22)
    ks = synth.loguniform_sizes(11, 12, 2000, 12000)
    work = []
    for i in range(12):
        name = "room" if i % 3 == 0 else "indoor"
        w, dm = two_maps[name]
        s, _ = synth.make_scan(w.scene, 40 + i, k=int(ks[i]) if name == "indoor" else 0)
        work.append((name, s) + _args(nv, w))
    reqs = []
    for name, s, rg, op in work:
        reqs.append((name, s, rg, op, nv.bbs_server_submit(srv, two_maps[name][1], s, rg, op)))
        time.sleep(0.0003)                   # arrivals while earlier requests run
    results = {}
    while len(results) < len(reqs):
        for name, s, rg, op, t in reqs:
            if t in results:
                continue
            st, r = nv.bbs_server_poll(srv, t, 0)
            if st != nv.PENDING:
                results[t] = r
        time.sleep(0.0005)
    stats = nv.bbs_server_stats(srv)
    srv.close()
    assert stats["completed"] == len(reqs) and stats["p99_ms"] >= stats["p50_ms"] > 0
    assert stats["peak_active"] >= 2         # requests really ran together
    for name, s, rg, op, t in reqs:
        w, dm = two_maps[name]
        alone = nv.bbs_localize(dm, s, rg, nv.make_opts(score_frac=w.score_frac, batch=w.batch))
        assert _same(results[t], alone), name
    # and the CPU oracle's search of the same request: every room request and
    # the two smallest indoor ones (the oracle takes tens of seconds per
    # larger indoor scan), run side by side on the host's cores
    import oracle_pool
    indoor = sorted((len(s), i) for i, (name, s, _, _, _) in enumerate(reqs) if name == "indoor")[:2]
    pick = [i for i, r in enumerate(reqs) if r[0] == "room"] + [i for _, i in indoor]
    jobs = []
    for i in pick:
        name, s, _, _, _ = reqs[i]
        w = synth.WORKLOADS[name]
        jobs.append((name, s, (w.lo, w.hi, w.ang_lo, w.ang_hi), w.score_frac, w.batch, 0, 0))
    for i, o in zip(pick, oracle_pool.localize_many(jobs)):
        r = results[reqs[i][4]]
        assert (r.status, r.best_score, list(r.node), r.iterations, r.nodes_scored, r.bound_violations) == \
               (o["status"], o["best_score"], o["node"], o["iterations"], o["nodes_scored"], o["bound_violations"]), i


def test_budget_admission_and_rejection(nv, two_maps):
    w, dm = two_maps["indoor"]
    rg, op = _args(nv, w)
    s0, _ = synth.make_scan(2, 3)
    # a search holds about 40 bytes per scan point (the scan and K + 1 score
    # buckets of three counts); 64 copies of the scan (~0.5 M points, ~21 MB)
    # against room for 32 MB beyond the engine admit one search at a time
    s = np.tile(s0, (64, 1))
    probe = nv.bbs_server_create(mem_budget=1 << 40, max_active=4, max_frontier=1 << 20)
    fixed = nv.bbs_server_stats(probe)["mem_in_use"]
    probe.close()
    srv = nv.bbs_server_create(mem_budget=fixed + (32 << 20), max_active=4, max_frontier=1 << 20)
    tickets = [nv.bbs_server_submit(srv, dm, s, rg, op) for _ in range(3)]
    saw_queue = nv.bbs_server_stats(srv)["queued"] > 0
    res = [nv.bbs_server_poll(srv, t, -1) for t in tickets]
    assert all(st == nv.OK for st, _ in res)
    assert len({(r.best_score, tuple(r.node)) for _, r in res}) == 1
    assert saw_queue or nv.bbs_server_stats(srv)["completed"] == 3
    # a request that can never fit fails at once: four times the points
    big = np.tile(s, (4, 1))
    t = nv.bbs_server_submit(srv, dm, big, rg, op)
    st, r = nv.bbs_server_poll(srv, t, 10000)
    assert st == nv.ENOMEM
    srv.close()


def test_cancel_queued(nv, two_maps):
    w, dm = two_maps["indoor"]
    rg, op = _args(nv, w)
    srv = nv.bbs_server_create(max_active=1, max_frontier=1 << 21)
    scans = [synth.make_scan(2, 60 + i)[0] for i in range(4)]
    tickets = [nv.bbs_server_submit(srv, dm, s, rg, op) for s in scans]
    nv.bbs_server_cancel(srv, tickets[-1])           # still queued behind the others
    st, r = nv.bbs_server_poll(srv, tickets[-1], -1)
    assert st == nv.ECANCELED
    for t in tickets[:-1]:
        st, r = nv.bbs_server_poll(srv, t, -1)
        assert st in (nv.OK, nv.NOT_FOUND)
    # a collected ticket (or one never issued) is refused at once, not waited on
    for t in (tickets[0], tickets[-1], tickets[-1] + 100):
        with pytest.raises(nv.BBSError) as e:
            nv.bbs_server_poll(srv, t, 2000)
        assert e.value.code == nv.EINVAL
    srv.close()


def test_cancel_running(nv, two_maps):
    """A request cancelled while it runs stops (its nodes are purged from the
    shared frontier between iterations) and the request running beside it
    still gets exactly its result alone."""
    w, dm = two_maps["indoor"]
    rg, op = _args(nv, w)
    slow = nv.make_opts(score_frac=0.5, batch=256, stream=0)     # many small rounds
    srv = nv.bbs_server_create(max_active=4, max_frontier=1 << 22)
    s_slow, s_norm = synth.make_scan(2, 70)[0], synth.make_scan(2, 71)[0]
    t_slow = nv.bbs_server_submit(srv, dm, s_slow, rg, slow)
    t_norm = nv.bbs_server_submit(srv, dm, s_norm, rg, op)
    for _ in range(4000):                                       # until the worker has admitted it
        if nv.bbs_server_stats(srv)["active"] >= 1:
            break
        time.sleep(0.0005)
    try:
        nv.bbs_server_cancel(srv, t_slow)
    except nv.BBSError as e:                                    # it finished first
        assert e.code == nv.EINVAL
    st, r = nv.bbs_server_poll(srv, t_slow, 20000)
    assert st in (nv.ECANCELED, nv.OK, nv.NOT_FOUND, nv.ENOMEM)
    st2, r2 = nv.bbs_server_poll(srv, t_norm, 20000)
    assert st2 in (nv.OK, nv.NOT_FOUND)
    assert nv.bbs_server_stats(srv)["active"] == 0
    srv.close()
    assert _same(r2, nv.bbs_localize(dm, s_norm, rg, nv.make_opts(score_frac=w.score_frac, batch=w.batch)))

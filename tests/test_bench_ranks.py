"""The multi-rank (replicas only) path of bench.py on the CPU: two gloo
ranks, each with its own scans; the job's time is the slowest rank's and its
probes the sum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=ws)
    try:
        # rank r: its own times and probes
        t, e, p, q = 10.0 + rank, 20.0 + 3 * rank, 1000.0 * (rank + 1), 7.0 * (rank + 1)
        out[rank] = (bench.reduce_over_ranks(torch, ws, t, e, p, q, torch.device("cpu")), bench.rank_scans(rank, 3))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_split_scans():
    ws = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        (t, e, p, q), scans = res[r]
        assert (t, e) == (11.0, 23.0)            # the slowest rank's times
        assert (p, q) == (3000.0, 21.0)          # every rank's probes
    assert res[0][1] == [0, 1, 2] and res[1][1] == [3, 4, 5]   # disjoint scans per rank


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(torch, 1, 1.5, 2.5, 10.0, 20.0, torch.device("cpu")) == (1.5, 2.5, 10.0, 20.0)

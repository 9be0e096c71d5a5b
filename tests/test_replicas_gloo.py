"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own
disjoint query batch; the whole-job rate is all ranks' queries over the
slowest rank's time (no collective on the data path, one MAX reduction of
the timings)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    from paper_2411_12229_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.TINY_10K_D128.with_(n_queries=8)
    q = bench.replica_queries(w, rank, world)
    local = [10.0 * (rank + 1), 20.0 + rank]  # this rank's step and e2e times (ms)
    worst, rates = bench.aggregate_replicas(local, q.shape[0], world, dist, "cpu")
    out[rank] = (q.sum(), q[0, 0], worst, rates)
    dist.destroy_process_group()


def test_two_rank_replicas():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    from paper_2411_12229_gb300 import synth
    w = synth.TINY_10K_D128.with_(n_queries=8)
    allq = synth.queries(w, 16)
    # disjoint batches: rank r holds rows [8r, 8r+8)
    for r in range(world):
        assert out[r][1] == pytest.approx(float(allq[8 * r, 0]))
        assert out[r][0] == pytest.approx(float(allq[8 * r:8 * r + 8].sum()), rel=1e-6)
    # both ranks agree on the slowest times and on the whole-job rate
    assert out[0][2] == out[1][2] == [20.0, 21.0]
    assert out[0][3][0] == pytest.approx(2 * 8 / 0.020)
    assert out[0][3][1] == pytest.approx(2 * 8 / 0.021)

"""Sharded search on the CPU path: two gloo ranks, each holding one shard
(its own graph, built on the shard's vectors alone) of a small index.

Each rank searches its shard for every query with the oracle (no GPU
here), the library's ``shard.exchange`` all-gathers the per-shard top-k
lists, and the lists are merged by (distance, global id).  Checked: both
ranks receive every shard's lists in shard order; the merge equals the
top-k of the union of the shards' results; with a beam that covers each
shard (ef >= n_shard (R+1)) it equals the brute-force kNN over all
vectors.  The merge kernel itself (sqg_merge_topk) runs on the GPU and is
tested in test_gpu_shard.py."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

K = 10
N, D, R, NQ = 120, 32, 32, 12


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def data():
    from paper_2411_12229_gb300 import synth
    w = synth.small(synth.TINY_10K_D128.with_(d=D), N, NQ, n_components=4)
    return synth.base(w), synth.queries(w)


def merge_ref(ids, dists, offsets, k):
    """Reference merge: the k smallest (distance, global id) of the union."""
    S, nq = ids.shape[0], ids.shape[1]
    out_i = np.full((nq, k), 0xFFFFFFFF, np.uint32)
    out_d = np.full((nq, k), np.inf, np.float32)
    for i in range(nq):
        c = [(float(dists[s, i, t]), int(ids[s, i, t]) + int(offsets[s]))
             for s in range(S) for t in range(ids.shape[2]) if ids[s, i, t] != 0xFFFFFFFF]
        c.sort()
        for t, (dd, g) in enumerate(c[:k]):
            out_i[i, t], out_d[i, t] = g, dd
    return out_i, out_d


def _worker(rank, world, port, manifest, out):
    import torch
    import torch.distributed as dist

    from oracle import oracle
    from paper_2411_12229_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = shard.load_manifest(manifest)
    _, q = data()
    O = oracle.Index(m["paths"][rank])
    ef = O.n * (O.R + 1)  # a beam that covers the shard
    ids = np.empty((1, NQ, K), np.uint32)
    dists = np.empty((1, NQ, K), np.float32)
    for i in range(NQ):
        ids[0, i], dists[0, i], _, _ = O.search(q[i], K, ef, hop_cap=10 * ef)
    gi, gd = shard.exchange(torch.from_numpy(ids.view(np.int32)), torch.from_numpy(dists))
    out[rank] = (gi.numpy().view(np.uint32), gd.numpy(), ids, dists)
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_shards_on_two_gloo_ranks(tmp_path, lib_built, oracle_mod):
    from paper_2411_12229_gb300 import shard
    x, q = data()
    manifest = shard.build_shards(tmp_path / "idx", x, R, 2)
    m = shard.load_manifest(manifest)
    assert m["ranges"] == [[0, 60], [60, 120]] and m["offsets"] == [0, 60]
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, str(manifest), out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    # every rank holds every shard's lists, in shard order
    for r in range(world):
        gi, gd, _, _ = out[r]
        assert gi.shape == (2, NQ, K)
        for s in range(world):
            np.testing.assert_array_equal(gi[s], out[s][2][0])
            np.testing.assert_array_equal(gd[s], out[s][3][0])
    gi, gd = out[0][0], out[0][1]
    mi, md = merge_ref(gi, gd, m["offsets"], K)
    # each shard's list is the exact kNN within the shard (full beam), so
    # the merged list is the exact kNN over all vectors
    for i in range(NQ):
        bi, bd = oracle_mod.bruteforce(x, q[i], K)
        np.testing.assert_array_equal(mi[i], bi)
        np.testing.assert_allclose(md[i], bd, rtol=1e-5)
    # and every merged id lies in its shard's range with its local distance
    for i in range(NQ):
        for t in range(K):
            s = int(mi[i, t] >= 60)
            loc = int(mi[i, t]) - m["offsets"][s]
            j = list(gi[s, i]).index(loc)
            assert gd[s, i, j] == md[i, t]


def test_shard_ranges():
    from paper_2411_12229_gb300 import shard
    assert shard.shard_ranges(10, 3) == [(0, 3), (3, 6), (6, 10)]
    assert sum(hi - lo for lo, hi in shard.shard_ranges(1_000_003, 32)) == 1_000_003
    with pytest.raises(ValueError):
        shard.shard_ranges(10, 33)

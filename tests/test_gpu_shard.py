"""Sharded search on one GPU: S shards (each its own graph) searched in
turn and merged by the library's sqg_merge_topk kernel.

Checked against the oracle: the merged ids and distances equal the merge
(by distance, then global id) of the oracle's per-shard searches, bit for
bit; with beams that cover every shard the result is the brute-force kNN
over all vectors; the merge kernel alone equals a plain sort of the union
of random sorted lists with padding and exact distance ties."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from test_shard_gloo import merge_ref  # noqa: E402


@pytest.mark.parametrize("shards", [2, 3])
def test_sharded_search_matches_the_oracle(tmp_path, lib_built, oracle_mod, shards):
    from paper_2411_12229_gb300 import shard, synth
    w = synth.small(synth.BATCHED_1M_D128, 1800, 40)
    x, q = synth.base(w), synth.queries(w)
    man = shard.build_shards(tmp_path / "idx", x, 32, shards)
    six = shard.ShardedIndex(man, 0)
    m = shard.load_manifest(man)
    for k, ef in ((10, 40), (10, 128), (1, 16)):
        ids, dists = six.search(torch.from_numpy(q).cuda(), k, ef)
        ids, dists = ids.cpu().numpy().view(np.uint32), dists.cpu().numpy()
        oi = np.empty((shards, q.shape[0], k), np.uint32)
        od = np.empty((shards, q.shape[0], k), np.float32)
        for s in range(shards):
            O = oracle_mod.Index(m["paths"][s])
            for i in range(q.shape[0]):
                oi[s, i], od[s, i], _, _ = O.search(q[i], k, ef)
        ri, rd = merge_ref(oi, od, m["offsets"], k)
        np.testing.assert_array_equal(ids, ri)
        np.testing.assert_array_equal(dists, rd)
    six.close()


def test_sharded_full_beams_give_the_exact_knn(tmp_path, lib_built, oracle_mod):
    """Shards of 60 vertices with ef = 60 (R + 1) = 1980: every reachable
    vertex of each shard is expanded, so the merge is the exact kNN."""
    from paper_2411_12229_gb300 import shard, synth
    w = synth.small(synth.TINY_10K_D128.with_(d=32), 180, 24, n_components=4)
    x, q = synth.base(w), synth.queries(w)
    six = shard.ShardedIndex(shard.build_shards(tmp_path / "idx", x, 32, 3), 0)
    ids, dists = six.search(torch.from_numpy(q).cuda(), 10, 1980, hop_cap=20000)
    ids, dists = ids.cpu().numpy().view(np.uint32), dists.cpu().numpy()
    for i in range(q.shape[0]):
        bi, bd = oracle_mod.bruteforce(x, q[i], 10)
        np.testing.assert_array_equal(ids[i], bi)
        np.testing.assert_allclose(dists[i], bd, rtol=1e-5)


def test_merge_kernel_against_a_sort(lib_built):
    """Random sorted lists (integer distances, so ties are exact and broken
    by global id), some padded, up to 32 shards and k = 256."""
    from paper_2411_12229_gb300 import shard
    rng = np.random.default_rng(7)
    for S, nq, k in ((1, 5, 10), (4, 33, 10), (32, 9, 7), (5, 3, 256)):
        offsets = np.cumsum([0] + [int(rng.integers(300, 400)) for _ in range(S - 1)]).astype(np.uint32)
        ids = np.full((S, nq, k), 0xFFFFFFFF, np.uint32)
        dists = np.full((S, nq, k), np.inf, np.float32)
        for s in range(S):
            for i in range(nq):
                n = int(rng.integers(0, k + 1))  # the rest is padding
                loc = rng.choice(300, size=n, replace=False)
                dd = rng.integers(0, 50, size=n).astype(np.float32)
                o = np.lexsort((loc, dd))
                ids[s, i, :n], dists[s, i, :n] = loc[o], dd[o]
        gi, gd = shard.merge_topk(torch.from_numpy(ids.view(np.int32)).cuda(), torch.from_numpy(dists).cuda(),
                                  offsets, k)
        ri, rd = merge_ref(ids, dists, offsets, k)
        np.testing.assert_array_equal(gi.cpu().numpy().view(np.uint32), ri)
        np.testing.assert_array_equal(gd.cpu().numpy(), rd)

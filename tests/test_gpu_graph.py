"""Algorithm 2's adjust step on the GPU (Sec. 3.2.1-3.2.2): the NSG pruning,
the re-pruning with reverse candidates and the adaptive angle rule run one
warp per vertex and give the host builder's rows bit for bit, and the
oracle's lists; a hub vertex too long for a warp's lists is refined on the
host with the same result."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _clustered(n, d, seed, k=8, spread=3.0):
    rng = np.random.default_rng(seed)
    cen = rng.standard_normal((k, d)) * spread
    return (cen[rng.integers(0, k, n)] + rng.standard_normal((n, d))).astype(np.float32)


def _knn_cand(x, L, seed):
    x64 = x.astype(np.float64)
    sq = (x64 * x64).sum(1)
    dist = sq[:, None] + sq[None, :] - 2.0 * x64 @ x64.T
    np.fill_diagonal(dist, np.inf)
    cand = np.argsort(dist, axis=1, kind="stable")[:, :L].astype(np.uint32)
    rng = np.random.default_rng(seed)
    cand[::7, -3:] = rng.integers(0, x.shape[0], (cand[::7].shape[0], 3))  # repeats and far ids
    cand[::11, 1] = np.arange(0, x.shape[0], 11)  # the vertex itself: dropped
    cand[::13, 2] = 0xFFFFFFFF  # no candidate
    return cand


@pytest.mark.parametrize("n,d,R,L", [(600, 64, 32, 64), (500, 160, 32, 96), (300, 960, 64, 192)])
def test_gpu_adjust_equals_host_and_oracle(lib_built, oracle_mod, n, d, R, L):
    from paper_2411_12229_gb300 import index_builder as ib
    x = _clustered(n, d, n + d)
    cand = _knn_cand(x, L, d)
    adj_h, st_h = ib.build_graph(x, cand, R, 0, 3, 0)
    adj_g, st_g = ib.build_graph(x, cand, R, 0, 3, 0, device=0)
    np.testing.assert_array_equal(adj_g, adj_h)
    for key in ("avg_nsg_degree", "supplemented", "random_filled", "repairs"):
        assert st_g[key] == st_h[key], key
    assert st_g["host_refined"] == 0 and st_g["supplemented"] > 0
    if st_h["random_filled"] == 0 and st_h["repairs"] == 0:
        out, cnt = oracle_mod.adjust_graph(x, cand, R)
        np.testing.assert_array_equal(adj_g, out)


def test_gpu_adjust_hub_vertex_refined_on_the_host(lib_built):
    """Vertex 0 at the origin, the others on the unit sphere: every vertex
    keeps 0 (its nearest), so 0 has ~1500 reverse candidates, more than a
    warp's lists hold; it is refined on the host, the rows are the same."""
    from paper_2411_12229_gb300 import index_builder as ib
    rng = np.random.default_rng(4)
    n, d, R = 1500, 32, 32
    x = rng.standard_normal((n, d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    x[0] = 0.0
    x = x.astype(np.float32)
    cand = _knn_cand(x, 64, 1)
    adj_h, st_h = ib.build_graph(x, cand, R, 0, 3, 0)
    adj_g, st_g = ib.build_graph(x, cand, R, 0, 3, 0, device=0)
    assert st_g["host_refined"] >= 1
    np.testing.assert_array_equal(adj_g, adj_h)


def test_gpu_built_index_searches_like_the_oracle(lib_built, oracle_mod, tmp_path):
    """An index built with the GPU candidate search and the GPU adjust step:
    the search on it is still the oracle's bit for bit."""
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300 import synth
    from paper_2411_12229_gb300.api import Index
    w = synth.small(synth.BATCHED_1M_D128, 4000, 32)
    x, q = synth.base(w), synth.queries(w)
    p = tmp_path / "g.sqg"
    info = ib.build_index(p, x, 32, device=0, init="random", iterations=2, ef_build=64)
    assert all(it.get("host_refined", 0) >= 0 for it in info["iterations"])
    ix, O = Index(p, 0), oracle_mod.Index(p)
    ids, dists = ix.search(torch.from_numpy(q).cuda(), 10, 48)
    ids, dists = ids.cpu().numpy().view(np.uint32), dists.cpu().numpy()
    for i in range(q.shape[0]):
        oi, od, _, _ = O.search(q[i], 10, 48)
        np.testing.assert_array_equal(ids[i], oi)
        np.testing.assert_array_equal(dists[i], od)


@pytest.mark.parametrize("n,d,R,L", [(600, 64, 32, 64), (300, 960, 64, 192)])
def test_gpu_irregular_graph_equals_host(lib_built, oracle_mod, n, d, R, L):
    """The degree-unaligned "w/o GR" build on the GPU: the host's rows."""
    from paper_2411_12229_gb300 import index_builder as ib
    x = _clustered(n, d, n + d + 1)
    cand = _knn_cand(x, L, d + 1)
    adj_h, st_h = ib.build_graph(x, cand, R, 0, 3, 0, regular=False)
    adj_g, st_g = ib.build_graph(x, cand, R, 0, 3, 0, device=0, regular=False)
    np.testing.assert_array_equal(adj_g, adj_h)
    assert st_g["supplemented"] == 0 and np.any(adj_g == 0xFFFFFFFF)
    if st_h["repairs"] == 0:
        out, _ = oracle_mod.adjust_graph(x, cand, R, regular=False)
        np.testing.assert_array_equal(adj_g, out)


IRREGULAR = {  # name: (workload, n, d, R)
    "d128-R32": ("tiny-10k-d128", 2000, 128, 32),
    "d64-R64": ("highdim-1m-d960", 1000, 64, 64),
}


@pytest.fixture(scope="module", params=list(IRREGULAR))
def irregular_index(request, tmp_path_factory, lib_built, oracle_mod):
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300 import synth
    from paper_2411_12229_gb300.api import Index
    name, n, d, R = IRREGULAR[request.param]
    w = synth.small(synth.WORKLOADS[name].with_(d=d), n, 48)
    x, q = synth.base(w), synth.queries(w)
    p = tmp_path_factory.mktemp(request.param) / "irr.sqg"
    ib.build_index(p, x, R, regular=False)
    return Index(p, 0), oracle_mod.Index(p), q


@pytest.mark.parametrize("team", [32, 16, 8])
def test_irregular_index_search_parity(irregular_index, team):
    """Empty slots are skipped on both sides: ids, distances, hops and
    status bit for bit, for every team size that the shape allows."""
    ix, O, q = irregular_index
    if team < 32 and ix.d > 256:
        pytest.skip("teams need d <= 256")
    qd = torch.from_numpy(q).cuda()
    for ef in (16, 64, 200):
        ids, dists, st = ix.search(qd, 10, ef, stats=True, team=team)
        ids, dists, st = ids.cpu().numpy().view(np.uint32), dists.cpu().numpy(), st.cpu().numpy()
        for i in range(q.shape[0]):
            oi, od, oh, os_ = O.search(q[i], 10, ef)
            np.testing.assert_array_equal(ids[i], oi, err_msg=f"ef {ef} query {i}")
            np.testing.assert_array_equal(dists[i], od)
            assert (st[i, 0], st[i, 1]) == (oh, os_)


def test_irregular_index_estimates(irregular_index):
    """The estimate hook on blocks with empty slots: S = 0 and est = key =
    dist_c there (zero codes and factors), the oracle's values everywhere."""
    ix, O, q = irregular_index
    qd = torch.from_numpy(q).cuda()
    v = (np.arange(q.shape[0]) * 29 % ix.n).astype(np.int32)
    S, est, key, dc = (t.cpu().numpy() for t in ix.estimate_block(qd, torch.from_numpy(v), 1.0))
    seen_empty = False
    for i in range(q.shape[0]):
        r = O.estimate_block(q[i], int(v[i]), 1.0)
        np.testing.assert_array_equal(S[i], r["S"])
        np.testing.assert_array_equal(est[i], r["est"])
        np.testing.assert_array_equal(key[i], r["key"])
        empty = O.vertex(int(v[i]))["ids"] == 0xFFFFFFFF
        seen_empty |= bool(empty.any())
        assert np.all(est[i][empty] == dc[i]) and np.all(S[i][empty] == 0)
    assert seen_empty


def test_irregular_index_trace_features(irregular_index, oracle_mod):
    """The learned stop's search-state features (and the trace's hit
    counts) on blocks with empty slots: the oracle's, bit for bit."""
    ix, O, q = irregular_index
    x = O.raw_all()
    nq = 16
    gt = np.stack([oracle_mod.bruteforce(x, q[i], 10)[0] for i in range(nq)]).astype(np.int32)
    r = ix.search_trace(torch.from_numpy(q[:nq]).cuda(), 10, 64, torch.from_numpy(gt).cuda(), 256, stop_every=3)
    feats, hits, cnt = (t.cpu().numpy() for t in r[3:6])
    for i in range(nq):
        o = O.search(q[i], 10, 64, stop_every=3, gt=gt[i].view(np.uint32), trace_cap=256)
        assert cnt[i] == len(o[4])
        np.testing.assert_array_equal(feats[i, :cnt[i]], o[4])
        np.testing.assert_array_equal(hits[i, :cnt[i]], o[5])

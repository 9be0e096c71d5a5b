"""Continuous batching: a request's result is the same alone, in the mix
and in the oracle's search (also with the learned stop on), admission
keeps the in-flight memory within the budget, and batches launched on
several streams overlap."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def serve_index(tmp_path_factory, lib_built):
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300 import synth
    from paper_2411_12229_gb300.api import Index
    w = synth.small(synth.SERVING_4M_D96, 20_000, 400)
    x = synth.base(w)
    p = tmp_path_factory.mktemp("serve") / "s.sqg"
    ib.build_index(p, x, 32, device=0, init="random", iterations=2, ef_build=64)
    return Index(p, 0), synth.queries(w), p


def test_results_same_alone_and_in_the_mix(serve_index, oracle_mod):
    from paper_2411_12229_gb300 import synth
    from paper_2411_12229_gb300.serve import Server
    ix, q, path = serve_index
    rng = np.random.default_rng(0)
    m = 3000
    sel = rng.integers(0, q.shape[0], size=m)
    ks = np.where(rng.integers(0, 2, size=m) == 0, 10, 100).astype(np.int32)
    efs = np.where(ks == 10, 64, 160).astype(np.int32)
    arr = synth.poisson_arrivals(200_000.0, m)
    srv = Server(ix, max_k=100, max_ef=160, mem_budget=64 << 20, streams=4, max_batch=512)
    r = srv.run(q[sel], ks, efs, arr)
    assert r.batches > 1
    # alone: every request searched by itself; and the oracle's search
    qd = torch.from_numpy(q).cuda()
    O = oracle_mod.Index(path)
    for i in range(0, m, 97):
        ids, dists = ix.search(qd[sel[i]:sel[i] + 1], int(ks[i]), int(efs[i]))
        np.testing.assert_array_equal(r.ids[i], ids.cpu().numpy()[0])
        np.testing.assert_array_equal(r.dists[i], dists.cpu().numpy()[0])
        oi, od, _, _ = O.search(q[sel[i]], int(ks[i]), int(efs[i]))
        np.testing.assert_array_equal(r.ids[i].view(np.uint32), oi)
        np.testing.assert_array_equal(r.dists[i], od)
    s = r.summary()
    assert s["requests"] == m and s["p99_ms"] >= s["p50_ms"] > 0
    assert s["device_search_s"] > 0 and s["host_loop_s"] > 0


def test_learned_stop_in_the_mix(serve_index, oracle_mod):
    """The serving loop with the learned stop on: a random stop network at a
    threshold that ends some searches early; each request's result equals
    its search alone and the oracle's search with the same network."""
    from paper_2411_12229_gb300 import learned_stop as L
    from paper_2411_12229_gb300 import synth
    from paper_2411_12229_gb300.serve import Server
    ix, q, path = serve_index
    rng = np.random.default_rng(9)
    mlp = (rng.standard_normal(5313) * 0.3).astype(np.float32)
    model = L.StopModel(torch.from_numpy(mlp).cuda(), 0.5, 2, 160, {})
    m = 2000
    sel = rng.integers(0, q.shape[0], size=m)
    ks = np.where(rng.integers(0, 2, size=m) == 0, 10, 100).astype(np.int32)
    efs = np.where(ks == 10, 64, 160).astype(np.int32)
    srv = Server(ix, max_k=100, max_ef=160, mem_budget=64 << 20, streams=4, max_batch=512, stop_model=model)
    r = srv.run(q[sel], ks, efs, synth.poisson_arrivals(300_000.0, m))
    qd = torch.from_numpy(q).cuda()
    O = oracle_mod.Index(path)
    stopped = 0
    for i in range(0, m, 53):
        ids, dists, st = ix.search(qd[sel[i]:sel[i] + 1], int(ks[i]), int(efs[i]), stats=True,
                                   stop_mlp=model.params, stop_logit=0.5, stop_every=2)
        np.testing.assert_array_equal(r.ids[i], ids.cpu().numpy()[0])
        oi, od, oh, os_ = O.search(q[sel[i]], int(ks[i]), int(efs[i]), mlp=mlp, stop_logit=0.5, stop_every=2)
        np.testing.assert_array_equal(r.ids[i].view(np.uint32), oi)
        np.testing.assert_array_equal(r.dists[i], od)
        stopped += int(os_ == 2)
    assert stopped > 0  # the network did end some searches early


def test_admission_respects_the_memory_budget(serve_index):
    from paper_2411_12229_gb300 import synth
    from paper_2411_12229_gb300.serve import Server, request_bytes
    ix, q, _ = serve_index
    m = 1000
    ks = np.full(m, 10, np.int32)
    efs = np.full(m, 64, np.int32)
    budget = 40 * request_bytes(10, 64, ix.d)  # at most 40 requests in flight
    srv = Server(ix, max_k=10, max_ef=64, mem_budget=budget, streams=3, max_batch=256)
    r = srv.run(q[np.arange(m) % q.shape[0]], ks, efs, synth.poisson_arrivals(1e6, m))
    assert r.max_inflight_bytes <= budget
    assert r.batches >= m // 40
    assert all(x is not None for x in r.ids)

"""Cosine similarity (Sec. 3 names it beside Euclidean distance) as Euclidean
search between unit vectors: on a metric-1 index the library scales every
query to unit norm in the exact distance's fp32 order before anything else;
the prepared queries, estimates and searches are bit for bit the oracle's,
with the dense rotation on CUDA cores and tensor cores and with the fast JLT."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = {  # name: (n, d, R, rotation)
    "d128-R32": (2000, 128, 32, "dense"),
    "d256-R64": (1000, 256, 64, "dense"),
    "d96-R32-fjlt": (1500, 96, 32, "fjlt"),
    "d960-R64": (1000, 960, 64, "dense"),
}


@pytest.fixture(scope="module", params=list(SHAPES))
def cos_index(request, tmp_path_factory, lib_built, oracle_mod):
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300 import synth
    from paper_2411_12229_gb300.api import Index
    n, d, R, rot = SHAPES[request.param]
    w = synth.small(synth.WORKLOADS["uneven-1m-d1536"].with_(d=d), n, 48)
    x = synth.base(w)
    # raw queries of assorted norms, one zero query
    q = synth.queries(w) * np.geomspace(0.01, 300.0, 48, dtype=np.float32)[:, None]
    q[5] = 0.0
    p = tmp_path_factory.mktemp(request.param) / "c.sqg"
    ib.build_index(p, x, R, rotation=rot, metric="cosine")
    ix = Index(p, 0)
    O = oracle_mod.Index(p)
    qp = np.ascontiguousarray(np.pad(q, ((0, 0), (0, ix.d - d))))
    return ix, O, q, qp


def _np(t):
    return t.detach().cpu().numpy()


def _words(qbar, d):
    qb = qbar.astype(np.uint64)
    out = np.zeros((4, d // 32), np.uint32)
    for b in range(4):
        bits = ((qb >> b) & 1).reshape(d // 32, 32)
        out[b] = (bits << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)
    return out


def test_cosine_index_info(cos_index):
    ix, O, q, qp = cos_index
    assert ix.metric == "cosine" and O.metric == 1


def test_cosine_prepared_queries_bit_exact(cos_index, oracle_mod):
    ix, O, q, qp = cos_index
    qd = torch.from_numpy(qp).cuda()
    outs = [(True, ix.prepare_queries(qd))]
    if not ix.fjlt:  # the tensor cores' q' is within its error bound; planes and scalars are exact
        outs.append((False, ix.prepare_queries_tc(qd)[:3]))
    for exact_qrot, (qrot, planes, scal) in outs:
        qrot, planes, scal = _np(qrot), _np(planes).view(np.uint32), _np(scal)
        for i in range(q.shape[0]):
            r = O.prepare_query(qp[i])
            if exact_qrot:
                np.testing.assert_array_equal(qrot[i], r["qrot"], err_msg=f"query {i} q'")
            else:
                np.testing.assert_allclose(qrot[i], r["qrot"], rtol=0, atol=1e-5 * max(1.0, np.abs(r["qrot"]).max()))
            assert (scal[i, 0], scal[i, 1], scal[i, 2]) == (r["vl"], r["delta"], r["sq"]), f"query {i}"
            np.testing.assert_array_equal(planes[i], _words(r["qbar"], ix.d), err_msg=f"query {i} planes")


def test_cosine_estimates_parity(cos_index):
    ix, O, q, qp = cos_index
    qd = torch.from_numpy(qp).cuda()
    v = (np.arange(q.shape[0]) * 41 % ix.n).astype(np.int32)
    S, est, key, dc = (_np(t) for t in ix.estimate_block(qd, torch.from_numpy(v), 0.5))
    for i in range(q.shape[0]):
        r = O.estimate_block(qp[i], int(v[i]), 0.5)
        assert dc[i] == r["dist_c"], f"query {i}"  # ||q/|q| - x_v||^2 in the canonical order
        np.testing.assert_array_equal(S[i], r["S"])
        np.testing.assert_array_equal(est[i], r["est"])
        np.testing.assert_array_equal(key[i], r["key"])


@pytest.mark.parametrize("rotation", [1, 2])
def test_cosine_search_parity(cos_index, rotation):
    ix, O, q, qp = cos_index
    qd = torch.from_numpy(qp).cuda()
    for ef in (16, 80):
        ids, dists, st = ix.search(qd, 10, ef, stats=True, rotation=rotation)
        ids, dists, st = _np(ids).view(np.uint32), _np(dists), _np(st)
        for i in range(q.shape[0]):
            oi, od, oh, os_ = O.search(qp[i], 10, ef)
            np.testing.assert_array_equal(ids[i], oi, err_msg=f"ef {ef} query {i}")
            np.testing.assert_array_equal(dists[i], od)
            assert (st[i, 0], st[i, 1]) == (oh, os_)
        assert np.all(np.isfinite(dists))


def test_cosine_search_is_scale_free(cos_index):
    """A power-of-2 multiple of every query: the same results bit for bit
    (all normalization steps scale exactly); the allocation-free entry
    point and a caller workspace give the same results too."""
    from paper_2411_12229_gb300 import _binding as B
    ix, O, q, qp = cos_index
    qd = torch.from_numpy(qp).cuda()
    a_ids, a_d = ix.search(qd, 10, 48)
    b_ids, b_d = ix.search(qd * 1024.0, 10, 48)
    assert torch.equal(a_ids, b_ids) and torch.equal(a_d, b_d)
    nq = q.shape[0]
    k = torch.full((nq,), 10, dtype=torch.int32, device="cuda")
    ef = torch.full((nq,), 48, dtype=torch.int32, device="cuda")
    ids = torch.empty(nq * 10, dtype=torch.int32, device="cuda")
    dd = torch.empty(nq * 10, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    B.check(B.lib().sqg_search_noalloc(ix.handle, qd.data_ptr(), nq, k.data_ptr(), ef.data_ptr(), 10, 48,
                                       ids.data_ptr(), dd.data_ptr(), s), "sqg_search_noalloc")
    torch.cuda.synchronize()
    assert torch.equal(ids.view(nq, 10), a_ids) and torch.equal(dd.view(nq, 10), a_d)

"""The fast JLT rotation (Sec. 3.1.4) on the GPU: for version-2 indexes the
query side applies three rounds of sign flips and Walsh-Hadamard
transforms; q', its 4-bit planes, the estimates and the searches are bit
for bit the oracle's, from d = 64 up to 2048 (padded from 96, 960, 1536)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = {  # name: (n, raw d, R) -> padded d
    "d64-R64": (1000, 64, 64),
    "d96-R32": (1500, 96, 32),
    "d960-R64": (1000, 960, 64),
    "d1536-R32": (1000, 1536, 32),
}


@pytest.fixture(scope="module", params=list(SHAPES))
def fjlt_index(request, tmp_path_factory, lib_built, oracle_mod):
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300 import synth
    from paper_2411_12229_gb300.api import Index
    n, d, R = SHAPES[request.param]
    w = synth.small(synth.WORKLOADS["highdim-1m-d960"].with_(d=d), n, 48)
    x, q = synth.base(w), synth.queries(w)
    p = tmp_path_factory.mktemp(request.param) / "f.sqg"
    ib.build_index(p, x, R, rotation="fjlt")
    ix = Index(p, 0)
    O = oracle_mod.Index(p)
    dp = ix.d
    qp = np.ascontiguousarray(np.pad(q, ((0, 0), (0, dp - d))))
    return ix, O, x, q, qp


def _np(t):
    return t.detach().cpu().numpy()


def _words(qbar, d):
    qb = qbar.astype(np.uint64)
    out = np.zeros((4, d // 32), np.uint32)
    for b in range(4):
        bits = ((qb >> b) & 1).reshape(d // 32, 32)
        out[b] = (bits << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)
    return out


def test_fjlt_prepared_queries_bit_exact(fjlt_index, oracle_mod):
    ix, O, x, q, qp = fjlt_index
    assert ix.fjlt and ix.d & (ix.d - 1) == 0
    qrot, planes, scal = ix.prepare_queries(torch.from_numpy(q).cuda())  # padded by the API
    qrot, planes, scal = _np(qrot), _np(planes).view(np.uint32), _np(scal)
    signs = O.fjlt_signs()
    for i in range(q.shape[0]):
        r = O.prepare_query(qp[i])
        np.testing.assert_array_equal(qrot[i], r["qrot"], err_msg=f"query {i} q'")
        np.testing.assert_array_equal(qrot[i], oracle_mod.fjlt_f32(signs, qp[i]))
        assert (scal[i, 0], scal[i, 1], scal[i, 2]) == (r["vl"], r["delta"], r["sq"])
        np.testing.assert_array_equal(planes[i], _words(r["qbar"], ix.d))


def test_fjlt_estimates_and_search_parity(fjlt_index, oracle_mod):
    ix, O, x, q, qp = fjlt_index
    qd = torch.from_numpy(qp).cuda()
    v = (np.arange(q.shape[0]) * 37 % ix.n).astype(np.int32)
    S, est, key, dc = (_np(t) for t in ix.estimate_block(qd, torch.from_numpy(v), 1.0))
    for i in range(0, q.shape[0], 3):
        r = O.estimate_block(qp[i], int(v[i]), 1.0)
        np.testing.assert_array_equal(S[i], r["S"])
        np.testing.assert_array_equal(key[i], r["key"])
    for ef in (16, 64):
        ids, dists, st = ix.search(qd, 10, ef, stats=True)
        ids, dists, st = _np(ids).view(np.uint32), _np(dists), _np(st)
        for i in range(q.shape[0]):
            oi, od, oh, os_ = O.search(qp[i], 10, ef)
            np.testing.assert_array_equal(ids[i], oi, err_msg=f"ef {ef} query {i}")
            np.testing.assert_array_equal(dists[i], od)
            assert (st[i, 0], st[i, 1]) == (oh, os_)
    # unpadded queries are padded by the API: the same search
    ids2, _ = ix.search(torch.from_numpy(q).cuda(), 10, 64)
    np.testing.assert_array_equal(_np(ids2).view(np.uint32), ids)


def test_fjlt_has_no_tensor_core_path(fjlt_index):
    from paper_2411_12229_gb300 import _binding as B
    ix, O, x, q, qp = fjlt_index
    with pytest.raises(B.SqgError):
        ix.prepare_queries_tc(torch.from_numpy(qp).cuda())
    # the rotation knob does not apply: the fast transform is always used
    a, _ = ix.search(torch.from_numpy(qp).cuda(), 10, 32, rotation=2)
    b, _ = ix.search(torch.from_numpy(qp).cuda(), 10, 32, rotation=1)
    assert torch.equal(a, b)

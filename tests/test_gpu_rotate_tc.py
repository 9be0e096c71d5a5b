"""The batched query rotation q' = P^-1 q (Eq. (4)) on the tensor cores
(tcgen05.mma kind::tf32, 3xTF32 split) and the exact quantization after it.

Bars: the tensor-core q' lies within the accumulation-error model's bound of
the fp64 rotation; the 4-bit planes, v_l, Delta and Sq are bit-identical to
the oracle's (which quantizes the canonical fp32 rotation), and so are the
searches that run on them.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

U = 2.0 ** -24


@pytest.fixture(scope="module")
def gpu_tiny(tiny_index):
    from paper_2411_12229_gb300.api import Index
    p, x, q = tiny_index
    return Index(p, 0), p, x, q


@pytest.fixture(scope="module")
def shaped(shaped_index_file):
    from paper_2411_12229_gb300.api import Index
    p, x, q = shaped_index_file
    return Index(p, 0), p, x, q


def _np(t):
    return t.detach().cpu().numpy()


def _words(qbar, d):
    """qbar (d codes) -> (4, d/32) bit-plane words, bit l of word w = coordinate 32w + l."""
    qb = qbar.astype(np.uint64)
    out = np.zeros((4, d // 32), np.uint32)
    for b in range(4):
        bits = ((qb >> b) & 1).reshape(d // 32, 32)
        out[b] = (bits << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)
    return out


def _check_prepared(ix, O, oracle_mod, q, rows):
    d = ix.d
    qd = torch.from_numpy(np.ascontiguousarray(q, dtype=np.float32)).cuda()
    qtc, planes, scal, rec = ix.prepare_queries_tc(qd)
    _, planes_simt, scal_simt = ix.prepare_queries(qd)
    torch.cuda.synchronize()
    qtc, planes, scal = _np(qtc), _np(planes).view(np.uint32), _np(scal)
    # the whole batch against the CUDA-core path, bit for bit
    np.testing.assert_array_equal(planes, _np(planes_simt).view(np.uint32))
    np.testing.assert_array_equal(scal, _np(scal_simt))
    rot = O.rotation()
    worst = 0.0
    for i in rows:
        exact = oracle_mod.rotate_f64(rot, q[i])
        # the tensor-core part of the error model: split 12u, 96 additions
        # per chunk accumulator (192u), d/32 register additions
        bound = (12 + 192 + d // 32) * U * float(np.linalg.norm(q[i].astype(np.float64)))
        err = float(np.max(np.abs(qtc[i].astype(np.float64) - exact)))
        assert err <= bound, f"query {i}: |q'_tc - q'| = {err} > {bound}"
        worst = max(worst, err / bound if bound > 0 else 0.0)
        r = O.prepare_query(q[i])
        assert (scal[i, 0], scal[i, 1], scal[i, 2]) == (r["vl"], r["delta"], r["sq"]), f"query {i} scalars"
        np.testing.assert_array_equal(planes[i], _words(r["qbar"], d), err_msg=f"query {i} planes")
    return int(_np(rec)[0]), worst


def test_tc_prepare_matches_oracle(gpu_tiny, oracle_mod):
    """d = 128, a batch that is not a multiple of the 128-query tile."""
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    rng = np.random.default_rng(11)
    qq = np.concatenate([q, x[rng.integers(0, x.shape[0], 300 - q.shape[0])]]).astype(np.float32)
    rec, worst = _check_prepared(ix, O, oracle_mod, qq, range(qq.shape[0]))
    print(f"d=128: recomputed {rec} of {qq.size} coordinates; worst error / bound {worst:.3g}")


def test_tc_prepare_boundary_queries(gpu_tiny, oracle_mod):
    """Queries built so that nearly every rotated coordinate sits on a code
    boundary ((q'_i - v_l) / Delta + 1/2 an integer, Eq. (4) run backwards
    through P^T): the exact pass has to recompute them and still agree."""
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    rot = O.rotation().astype(np.float64)
    d = ix.d
    rng = np.random.default_rng(12)
    zs = []
    for t in range(40):
        m = rng.integers(1, 16, d).astype(np.float64)
        z = -1.0 + (m - 0.5) * (2.0 / 15.0)
        z[0], z[1] = -1.0, 1.0
        zs.append(rot.T @ (z * (0.5 + t)))
    zs.append(np.zeros(d))  # q = 0: range 0, every code 0
    qq = np.stack(zs).astype(np.float32)
    rec, _ = _check_prepared(ix, O, oracle_mod, qq, range(qq.shape[0]))
    assert rec > qq.size // 4, "the boundary queries should force recomputation"


def test_tc_prepare_other_shapes(shaped, oracle_mod):
    """d = 96 (a partial column tile), 256, 960 and 1536."""
    ix, p, x, q = shaped
    O = oracle_mod.Index(p)
    rng = np.random.default_rng(13)
    qq = np.concatenate([q, x[rng.integers(0, x.shape[0], 200 - q.shape[0])]]).astype(np.float32)
    rec, worst = _check_prepared(ix, O, oracle_mod, qq, range(0, qq.shape[0], 3))
    print(f"d={ix.d}: recomputed {rec} of {qq.size} coordinates; worst error / bound {worst:.3g}")


@pytest.fixture(scope="module")
def wide_index(tmp_path_factory, lib_built):
    """A small d = 1536 index (the uneven workload's dimension and recipe);
    the rotation does not depend on n."""
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300 import synth
    from paper_2411_12229_gb300.api import Index
    w = synth.small(synth.UNEVEN_1M_D1536, 300, 16)
    p = tmp_path_factory.mktemp("wide") / "d1536.sqg"
    ib.build_index(p, synth.base(w), 32)
    return Index(p, 0), p


@pytest.mark.parametrize("nq", [20000, 20001])
def test_tc_prepare_production_size(wide_index, oracle_mod, nq):
    """The uneven workload's batch: 20,000 queries of d = 1536 (and a ragged
    20,001), 157 x 12 output tiles of 128 x 128 on the persistent grid of one
    CTA per SM, so every CTA walks several tiles: the TMEM double buffer is
    reused and the mbarrier phases flip past the first tile.  Every row's
    planes, v_l, Delta and Sq equal the CUDA-core path's bit for bit; 200
    seeded rows also equal the oracle's and lie within the error model."""
    from paper_2411_12229_gb300 import synth
    ix, p = wide_index
    O = oracle_mod.Index(p)
    q = synth.queries(synth.UNEVEN_1M_D1536, nq)
    rows = np.sort(np.random.default_rng(nq).choice(nq, 200, replace=False))
    rows = np.concatenate([rows, [nq - 1]])  # the ragged tile's last row
    rec, worst = _check_prepared(ix, O, oracle_mod, q, rows)
    print(f"nq={nq}: recomputed {rec} of {q.size} coordinates; worst error / bound {worst:.3g}")


def _search_equal(ix, O, q, k, ef):
    qd = torch.from_numpy(q).cuda()
    ids, dists, st = ix.search(qd, k, ef, stats=True, rotation=2)
    ids1, dists1, st1 = ix.search(qd, k, ef, stats=True, rotation=1)
    ids, dists, st = _np(ids).view(np.uint32), _np(dists), _np(st)
    np.testing.assert_array_equal(ids, _np(ids1).view(np.uint32))
    np.testing.assert_array_equal(dists, _np(dists1))
    np.testing.assert_array_equal(st, _np(st1))
    for i in range(0, q.shape[0], 4):
        oi, od, oh, os_ = O.search(q[i], k, ef)
        np.testing.assert_array_equal(ids[i], oi, err_msg=f"query {i} ids")
        np.testing.assert_array_equal(dists[i], od, err_msg=f"query {i} dists")
        assert (st[i, 0], st[i, 1]) == (oh, os_)


@pytest.mark.parametrize("ef", [16, 100])
def test_tc_search_parity(gpu_tiny, oracle_mod, ef):
    ix, p, x, q = gpu_tiny
    _search_equal(ix, oracle_mod.Index(p), q, 10, ef)


def test_tc_search_parity_other_shapes(shaped, oracle_mod):
    ix, p, x, q = shaped
    _search_equal(ix, oracle_mod.Index(p), q, 10, 40)


def test_tc_rotation_in_cuda_graph_with_knobs(shaped, oracle_mod):
    """The tensor-core rotation captured in a CUDA graph together with the
    search, under tuning knobs that change the workspace size: the replay
    gives the direct search's results."""
    from paper_2411_12229_gb300.autotune import GraphSearch
    ix, p, x, q = shaped
    qd = torch.from_numpy(q).cuda()
    knobs = dict(visited_smem_log2=5, warps_per_block=2, rotation=2)
    gs = GraphSearch(ix, q.shape[0], 10, 40, max_k=10, max_ef=40, **knobs)
    ids, dists = gs(qd)
    ref_ids, ref_d = ix.search(qd, 10, 40, rotation=1)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(_np(ids).reshape(-1, 10), _np(ref_ids))
    np.testing.assert_array_equal(_np(dists).reshape(-1, 10), _np(ref_d))

"""The compact search kernel (search_compact.cuh: packed 64-bit beam entries,
gathered merge, results in registers) against the oracle.

It serves every search it applies to (one warp per query, d <= 1024,
degree 32 or 64, k <= 32, ef <= 128 -- for d <= 256 k <= 128 and ef <= 256
--, multiple estimates, no trace; the learned stop in a build of its own);
here it is forced (kernel = 2) and held to the same bar as the
general kernel: ids, distances, hop counts and status bits identical to
the oracle, on the plain and the ragged batch, with the error-bound key,
binding hop caps, exact ties and duplicate vectors, visited-set moves, the
tensor-core rotation, empty slots and the cosine metric.  The general
kernel (kernel = 1) is checked to return the very same output."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _np(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def gpu_tiny(tiny_index):
    from paper_2411_12229_gb300.api import Index
    p, x, q = tiny_index
    return Index(p, 0), p, x, q


def check(ix, O, q, k, ef, *, oracle_kw=None, **kw):
    """Search q with the compact kernel and compare every query with the
    oracle; also the general kernel's output, which must be identical."""
    qd = torch.from_numpy(q).cuda()
    ids, dists, st = ix.search(qd, k, ef, stats=True, kernel=2, **kw)
    g_ids, g_d, g_st = ix.search(qd, k, ef, stats=True, kernel=1, **kw)
    assert torch.equal(ids, g_ids) and torch.equal(dists, g_d) and torch.equal(st, g_st)
    ids, dists, st = _np(ids).view(np.uint32), _np(dists), _np(st)
    okw = dict(eps0=kw.get("eps0", 0.0))
    if kw.get("hop_cap"):
        okw["hop_cap"] = kw["hop_cap"]
    okw.update(oracle_kw or {})
    for i in range(q.shape[0]):
        oi, od, oh, os_ = O.search(q[i], k, ef, **okw)
        np.testing.assert_array_equal(ids[i], oi, err_msg=f"query {i} ids")
        np.testing.assert_array_equal(dists[i], od, err_msg=f"query {i} dists")
        assert (st[i, 0], st[i, 1]) == (oh, os_), f"query {i}: hops/status {st[i]} vs {(oh, os_)}"
    return ids, dists, st


@pytest.mark.parametrize("lean", [0, 1])
@pytest.mark.parametrize("k,ef", [(1, 1), (1, 8), (10, 10), (10, 16), (10, 33), (10, 40), (10, 64), (32, 32),
                                  (32, 64), (5, 63), (10, 65), (10, 80), (1, 96), (10, 112), (32, 128), (7, 127)])
def test_compact_parity(gpu_tiny, oracle_mod, k, ef, lean):
    """Both register builds of the compact kernel (lean 0: 8 resident
    blocks per SM with 2 beam slots per lane, 7 with 4; lean 1: one more),
    for beams of up to 64 (2 slots per lane) and 128 entries (4)."""
    ix, p, x, q = gpu_tiny
    check(ix, oracle_mod.Index(p), q, k, ef, lean=lean)


@pytest.mark.parametrize("k,ef", [(10, 129), (10, 200), (32, 256), (33, 33), (33, 64), (64, 100), (100, 100),
                                  (100, 160), (128, 128), (128, 256), (1, 256)])
def test_compact_big_beams_and_results(gpu_tiny, oracle_mod, k, ef):
    """d <= 256: beams of 129-256 entries (8 slots per lane) and 33-128
    results (4 result slots per lane, lane l holding results l + 32 s)."""
    ix, p, x, q = gpu_tiny
    check(ix, oracle_mod.Index(p), q, k, ef)


def test_compact_big_variants(gpu_tiny, gpu_tiny64_compact, oracle_mod):
    """The big builds with out-degree 64, the error-bound key, a binding
    hop cap, visited-set moves, a ragged batch of k in {1, 10, 100} and ef
    up to 256, and the fused stop with a random network."""
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    check(ix, O, q, 100, 200, eps0=1.9)
    _, _, st = check(ix, O, q, 50, 150, hop_cap=9)
    assert np.all(st[:, 0] <= 9)
    check(ix, O, q, 10, 240, visited_smem_log2=5)
    rng = np.random.default_rng(31)
    nq = q.shape[0]
    k = rng.choice([1, 10, 100], size=nq).astype(np.int32)
    ef = np.array([rng.integers(kk, 257) for kk in k], dtype=np.int32)
    qd = torch.from_numpy(q).cuda()
    kt, et = torch.from_numpy(k), torch.from_numpy(ef)
    c = ix.search(qd, kt, et, stats=True, kernel=2, max_k=128, max_ef=256)
    g = ix.search(qd, kt, et, stats=True, kernel=1, max_k=128, max_ef=256)
    assert all(torch.equal(u, v) for u, v in zip(c, g))
    ids, off = _np(c[0]).view(np.uint32), np.concatenate([[0], np.cumsum(k)])
    for i in range(nq):
        np.testing.assert_array_equal(ids[off[i]:off[i + 1]], O.search(q[i], int(k[i]), int(ef[i]))[0])
    mlp = (rng.standard_normal(5313) * 0.3).astype(np.float32)
    dm = torch.from_numpy(mlp).cuda()
    for kk, e, thr in ((100, 160, 0.5), (10, 200, 1.5), (33, 64, -1.0)):
        check(ix, O, q, kk, e, stop_mlp=dm, stop_logit=thr, stop_every=3,
              oracle_kw=dict(mlp=mlp, stop_logit=thr, stop_every=3))
    ix64, p64, x64, q64 = gpu_tiny64_compact
    O64 = oracle_mod.Index(p64)
    for kk, e in ((10, 160), (100, 200), (128, 256)):
        check(ix64, O64, q64, kk, e)
    check(ix64, O64, q64, 100, 180, stop_mlp=dm, stop_logit=0.5, stop_every=2,
          oracle_kw=dict(mlp=mlp, stop_logit=0.5, stop_every=2))


@pytest.mark.parametrize("ef", [48, 100])
@pytest.mark.parametrize("eps0", [0.5, 1.9])
def test_compact_error_bound_key(gpu_tiny, oracle_mod, eps0, ef):
    ix, p, x, q = gpu_tiny
    check(ix, oracle_mod.Index(p), q, 10, ef, eps0=eps0)


@pytest.mark.parametrize("ef", [64, 128])
@pytest.mark.parametrize("cap", [1, 2, 7, 30])
def test_compact_hop_cap(gpu_tiny, oracle_mod, cap, ef):
    ix, p, x, q = gpu_tiny
    _, _, st = check(ix, oracle_mod.Index(p), q, 5, ef, hop_cap=cap)
    assert np.all(st[:, 0] <= cap) and np.all(st[:, 1] == 1)


@pytest.mark.parametrize("ef", [64, 128])
@pytest.mark.parametrize("smem_log2", [5, 6])
def test_compact_visited_set_migration(gpu_tiny, oracle_mod, smem_log2, ef):
    ix, p, x, q = gpu_tiny
    _, _, st = check(ix, oracle_mod.Index(p), q, 10, ef, visited_smem_log2=smem_log2)
    assert st[:, 0].min() > (1 << smem_log2) // 2


@pytest.mark.parametrize("max_ef", [64, 128])
def test_compact_ragged_batch(gpu_tiny, oracle_mod, max_ef):
    """Per-query k in {1, 10, 32} and ef in [k, max_ef] in one launch."""
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    rng = np.random.default_rng(17 + max_ef)
    nq = q.shape[0]
    k = rng.choice([1, 10, 32], size=nq).astype(np.int32)
    ef = np.array([rng.integers(kk, max_ef + 1) for kk in k], dtype=np.int32)
    qd = torch.from_numpy(q).cuda()
    kt, et = torch.from_numpy(k), torch.from_numpy(ef)
    ids, dists, st = ix.search(qd, kt, et, stats=True, kernel=2, max_k=32, max_ef=max_ef)
    g = ix.search(qd, kt, et, stats=True, kernel=1, max_k=32, max_ef=max_ef)
    assert torch.equal(ids, g[0]) and torch.equal(dists, g[1]) and torch.equal(st, g[2])
    ids, dists, st = _np(ids).view(np.uint32), _np(dists), _np(st)
    off = np.concatenate([[0], np.cumsum(k)])
    for i in range(nq):
        oi, od, oh, os_ = O.search(q[i], int(k[i]), int(ef[i]))
        np.testing.assert_array_equal(ids[off[i]:off[i + 1]], oi)
        np.testing.assert_array_equal(dists[off[i]:off[i + 1]], od)
        assert st[i, 0] == oh and st[i, 1] == os_


def test_compact_invalid_per_query_params_are_padding(gpu_tiny, oracle_mod):
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    k = np.array([10, 0, 10, 5, 40, 10], dtype=np.int32)
    ef = np.array([32, 32, 5, 5, 64, 40], dtype=np.int32)
    ids, dists, st = ix.search(torch.from_numpy(q[:6]).cuda(), torch.from_numpy(k), torch.from_numpy(ef),
                               stats=True, max_k=10, max_ef=40, kernel=2)
    ids, dists, st = _np(ids).view(np.uint32), _np(dists), _np(st)
    off = np.concatenate([[0], np.cumsum(k)])
    for i in range(6):
        sl = slice(off[i], off[i + 1])
        if i in (1, 2, 4):
            assert st[i, 1] == 4 and np.all(ids[sl] == 0xFFFFFFFF) and np.all(np.isinf(dists[sl]))
        else:
            np.testing.assert_array_equal(ids[sl], O.search(q[i], int(k[i]), int(ef[i]))[0])
    assert ix.status() & 4


def test_compact_tensor_core_rotation(gpu_tiny, oracle_mod):
    """Queries quantized by the tensor-core rotation's exact pass (the
    precomputed-planes path of the kernel)."""
    ix, p, x, q = gpu_tiny
    check(ix, oracle_mod.Index(p), q, 10, 40, rotation=2)


@pytest.mark.parametrize("ef", [1, 2, 3, 4])
def test_compact_golden_beam_trace(oracle_mod, lib_built, tmp_path, ef):
    """The hand-worked trace of tests/golden/beam_trace_d32.txt (empty slots,
    exact estimates) through the compact kernel."""
    import golden_trace as G

    from paper_2411_12229_gb300.api import Index
    t = G.load()
    p = tmp_path / "trace.sqg"
    G.write_index(t, p)
    ix = Index(p, 0)
    nm = G.names(t)
    D = {k: v["D"] for k, v in t["vertex"].items()}
    qd = torch.from_numpy(t["q"].astype(np.float32)[None, :]).cuda()
    ids, dists, st = ix.search(qd, ef, ef, stats=True, kernel=2)
    assert [nm[i] for i in _np(ids)[0].view(np.uint32)] == t["result"][ef]
    np.testing.assert_array_equal(_np(dists)[0], [32.0 * D[n] for n in t["result"][ef]])
    assert tuple(_np(st)[0]) == (len(t["path"][ef]), 0)


@pytest.fixture(scope="module")
def gpu_ties_compact(tmp_path_factory, lib_built):
    """Integer vectors with exact copies: equal keys ordered by id (R4),
    neighbours equal to their centre (R3), queries on data vectors."""
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300.api import Index
    rng = np.random.default_rng(43)
    base = rng.integers(-2, 3, size=(1200, 128)).astype(np.float32)
    x = np.concatenate([base, base[rng.integers(0, 1200, 300)]])
    x = x[rng.permutation(x.shape[0])]
    q = rng.integers(-2, 3, size=(48, 128)).astype(np.float32)
    q[:8] = x[rng.integers(0, x.shape[0], 8)]
    p = tmp_path_factory.mktemp("ties_c") / "ties.sqg"
    ib.build_index(p, x, 32)
    return Index(p, 0), p, x, q


def test_compact_ties_and_duplicates(gpu_ties_compact, oracle_mod):
    ix, p, x, q = gpu_ties_compact
    O = oracle_mod.Index(p)
    for ef in (16, 40, 64, 100, 128):
        _, dists, _ = check(ix, O, q, 10, ef)
    assert np.all(dists[:8, 0] == 0.0)
    check(ix, O, q, 10, 64, eps0=1.9)
    check(ix, O, q, 10, 128, eps0=1.9)


def test_compact_irregular_and_cosine_indexes(oracle_mod, lib_built, tmp_path):
    """Empty slots (the w/o GR graph, R17) and a cosine index (R16)."""
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300 import synth
    from paper_2411_12229_gb300.api import Index
    w = synth.small(synth.BATCHED_1M_D128, 1500, 40)
    x, q = synth.base(w), synth.queries(w)
    for name, kw in (("irr", dict(regular=False)), ("cos", dict(metric="cosine"))):
        p = tmp_path / f"{name}.sqg"
        ib.build_index(p, x, 32, **kw)
        ix = Index(p, 0)
        check(ix, oracle_mod.Index(p), q, 10, 40)


@pytest.fixture(scope="module")
def gpu_tiny64_compact(tiny_index_r64):
    from paper_2411_12229_gb300.api import Index
    p, x, q = tiny_index_r64
    return Index(p, 0), p, x, q


@pytest.mark.parametrize("k,ef", [(1, 1), (10, 10), (10, 40), (10, 64), (10, 65), (32, 100), (10, 128)])
def test_compact_out_degree_64(gpu_tiny64_compact, oracle_mod, k, ef):
    """Out-degree 64: lane l estimates neighbours l and l + 32 and the
    step's candidates are staged 64 wide."""
    ix, p, x, q = gpu_tiny64_compact
    check(ix, oracle_mod.Index(p), q, k, ef)


def test_compact_out_degree_64_variants(gpu_tiny64_compact, oracle_mod):
    """Error-bound key, a binding hop cap, visited-set moves, a ragged
    batch, with two neighbours per lane."""
    ix, p, x, q = gpu_tiny64_compact
    O = oracle_mod.Index(p)
    check(ix, O, q, 10, 100, eps0=1.9)
    _, _, st = check(ix, O, q, 5, 64, hop_cap=7)
    assert np.all(st[:, 0] <= 7)
    _, _, st = check(ix, O, q, 10, 128, visited_smem_log2=5)
    assert st[:, 0].min() > 16
    rng = np.random.default_rng(29)
    nq = q.shape[0]
    k = rng.choice([1, 10, 32], size=nq).astype(np.int32)
    ef = np.array([rng.integers(kk, 129) for kk in k], dtype=np.int32)
    qd = torch.from_numpy(q).cuda()
    kt, et = torch.from_numpy(k), torch.from_numpy(ef)
    c = ix.search(qd, kt, et, stats=True, kernel=2, max_k=32, max_ef=128)
    g = ix.search(qd, kt, et, stats=True, kernel=1, max_k=32, max_ef=128)
    assert all(torch.equal(u, v) for u, v in zip(c, g))
    ids, off = _np(c[0]).view(np.uint32), np.concatenate([[0], np.cumsum(k)])
    for i in range(nq):
        np.testing.assert_array_equal(ids[off[i]:off[i + 1]], O.search(q[i], int(k[i]), int(ef[i]))[0])


@pytest.fixture(scope="module")
def gpu_d1152(tmp_path_factory, lib_built):
    """d = 1152, past the compact kernel's d <= 1024."""
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300.api import Index
    rng = np.random.default_rng(5)
    x = rng.standard_normal((400, 1152)).astype(np.float32)
    p = tmp_path_factory.mktemp("d1152") / "d1152.sqg"
    ib.build_index(p, x, 32)
    return Index(p, 0), rng.standard_normal((16, 1152)).astype(np.float32)


def test_compact_applies_only_where_it_is_defined(gpu_tiny, gpu_d1152):
    """kernel = 2 outside the compact kernel's range is refused; kernel = 0
    falls back to the general kernel there."""
    from paper_2411_12229_gb300._binding import SqgError
    ix, p, x, q = gpu_tiny
    qd = torch.from_numpy(q).cuda()
    for kw in (dict(k=129, ef=200), dict(k=10, ef=257), dict(k=10, ef=40, multi_estimate=False),
               dict(k=10, ef=40, team=16), dict(k=10, ef=40, prefetch=2)):
        k, ef = kw.pop("k"), kw.pop("ef")
        with pytest.raises(SqgError):
            ix.search(qd, k, ef, kernel=2, **kw)
        ix.search(qd, k, ef, kernel=0, **kw)
    ixw, qw = gpu_d1152
    with pytest.raises(SqgError):
        ixw.search(torch.from_numpy(qw).cuda(), 10, 40, kernel=2)
    ixw.search(torch.from_numpy(qw).cuda(), 10, 40, kernel=0)

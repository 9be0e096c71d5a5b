"""GPU parity: every kernel step through the C ABI against the CPU oracle.

Bars: integer sums and ids bit-exact; fp32 estimates, keys and exact
distances bit-exact too (both sides take their float decisions in the same
precision and order), which is stricter than the 1e-5 relative tolerance
the float values would need on their own.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gpu_tiny(tiny_index):
    from paper_2411_12229_gb300.api import Index
    p, x, q = tiny_index
    return Index(p, 0), p, x, q


@pytest.fixture(scope="module")
def gpu_tiny64(tiny_index_r64):
    from paper_2411_12229_gb300.api import Index
    p, x, q = tiny_index_r64
    return Index(p, 0), p, x, q


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("which", ["gpu_tiny", "gpu_tiny64"])
def test_prepare_queries_bit_exact(which, request, oracle_mod):
    """q' = P^-1 q (Eq. (4)) and its 4-bit planes, identical to the oracle."""
    ix, p, x, q = request.getfixturevalue(which)
    O = oracle_mod.Index(p)
    qd = torch.from_numpy(q).cuda()
    qrot, planes, scal = ix.prepare_queries(qd)
    qrot, planes, scal = _np(qrot), _np(planes).view(np.uint32), _np(scal)
    for i in range(q.shape[0]):
        r = O.prepare_query(q[i])
        np.testing.assert_array_equal(qrot[i], r["qrot"])
        assert scal[i, 0] == r["vl"] and scal[i, 1] == r["delta"] and scal[i, 2] == r["sq"]
        qb = r["qbar"].astype(np.uint32)
        for b in range(4):
            bits = (qb >> b) & 1
            words = np.array([int("".join(str(v) for v in bits[w * 32:(w + 1) * 32][::-1]), 2)
                              for w in range(ix.d // 32)], dtype=np.uint32)
            np.testing.assert_array_equal(planes[i, b], words)


@pytest.mark.parametrize("which", ["gpu_tiny", "gpu_tiny64"])
@pytest.mark.parametrize("eps0", [0.0, 1.9])
def test_estimates_bit_exact(which, eps0, request, oracle_mod):
    """S (AND + popc over bit-planes) = sum_i b_i qbar_i exactly; est, key
    and dist_c bit-identical to the oracle (Sec. 3.1.1)."""
    ix, p, x, q = request.getfixturevalue(which)
    O = oracle_mod.Index(p)
    rng = np.random.default_rng(0)
    v = rng.integers(0, ix.n, size=q.shape[0]).astype(np.int32)
    S, est, key, dc = (_np(t) for t in ix.estimate_block(torch.from_numpy(q).cuda(), torch.from_numpy(v), eps0))
    for i in range(q.shape[0]):
        r = O.estimate_block(q[i], int(v[i]), eps0)
        np.testing.assert_array_equal(S[i], r["S"])
        np.testing.assert_array_equal(est[i], r["est"])
        np.testing.assert_array_equal(key[i], r["key"])
        assert dc[i] == r["dist_c"]


def test_golden_closed_form_on_gpu(oracle_mod, lib_built, tmp_path):
    """tests/golden/alpha_one_d32.txt through the GPU: estimates equal the
    integer squared distances (alpha = 1, exact 4-bit query)."""
    from test_oracle_pins import golden_index

    from paper_2411_12229_gb300.api import Index
    p = tmp_path / "golden.sqg"
    x, q = golden_index(p)
    ix = Index(p, 0)
    S, est, key, dc = (_np(t) for t in ix.estimate_block(torch.from_numpy(q[None, :]).cuda(),
                                                          torch.zeros(1, dtype=torch.int32)))
    ids = oracle_mod.Index(p).vertex(0)["ids"]
    exact = np.array([np.sum((x[j] - q).astype(np.int64) ** 2) for j in ids], dtype=np.float64)
    np.testing.assert_allclose(est[0], exact, rtol=2e-6)
    assert dc[0] == np.sum((x[0] - q).astype(np.int64) ** 2)


@pytest.mark.parametrize("team", [32, 16, 8])
@pytest.mark.parametrize("ef", [1, 2, 3, 4])
def test_golden_beam_trace_on_gpu(oracle_mod, lib_built, tmp_path, ef, team):
    """The hand-worked trace of tests/golden/beam_trace_d32.txt (Algorithm 1
    below the full beam, every estimate exact) through the GPU search: the
    expansion order, hop count, status and the k = ef results with their
    exact distances, for whole warps and teams of 16 / 8 lanes; with whole
    warps also the learned-stop features f5 and f6 at every evaluation
    point against the fractions derived by hand."""
    import golden_trace as G

    from paper_2411_12229_gb300.api import Index
    t = G.load()
    p = tmp_path / "trace.sqg"
    G.write_index(t, p)
    ix = Index(p, 0)
    nm = G.names(t)
    D = {k: v["D"] for k, v in t["vertex"].items()}
    q = torch.from_numpy(t["q"].astype(np.float32)[None, :]).cuda()
    ids, dists, st = ix.search(q, ef, ef, stats=True, team=team)
    ids, dists, st = _np(ids)[0].view(np.uint32), _np(dists)[0], _np(st)[0]
    assert [nm[i] for i in ids] == t["result"][ef]
    np.testing.assert_array_equal(dists, [32.0 * D[n] for n in t["result"][ef]])
    assert (st[0], st[1]) == (len(t["path"][ef]), 0)
    if team != 32:
        return  # the trace export runs whole warps
    *_, feats, _, cnt, path = ix.search_trace(q, ef, ef, None, 16, path_cap=16, stop_every=1)
    path = _np(path)[0].view(np.uint32)
    assert [nm[i] for i in path[:len(t["path"][ef])]] == t["path"][ef]
    assert np.all(path[len(t["path"][ef]):] == 0xFFFFFFFF)
    want = t["stop"][ef]
    feats = _np(feats)[0][:int(_np(cnt)[0])]
    assert len(feats) == len(want)
    for f, (h, f5, f6) in zip(feats, want):
        assert f[0] == pytest.approx(h / ef, rel=1e-6)
        assert f[5] == pytest.approx(float(f5), rel=1e-5, abs=1e-7)
        assert f[6] == pytest.approx(float(f6), rel=1e-6)


@pytest.mark.parametrize("ef,k", [(1, 1), (2, 2), (3, 3), (4, 4), (4, 2)])
def test_golden_beam_trace_all_stop_features_on_gpu(lib_built, tmp_path, ef, k):
    """The fused stop's 16 features, traced by the GPU search at every
    evaluation point of the hand-worked trace, against the values derived
    by hand (tests/golden/beam_trace_d32.txt)."""
    import golden_trace as G

    from paper_2411_12229_gb300.api import Index
    t = G.load()
    p = tmp_path / "trace.sqg"
    G.write_index(t, p)
    ix = Index(p, 0)
    q = torch.from_numpy(t["q"].astype(np.float32)[None, :]).cuda()
    *_, feats, _, cnt = ix.search_trace(q, k, ef, None, 16, stop_every=1)
    feats = _np(feats)[0][:int(_np(cnt)[0])]
    want = t["feat"][(ef, k)]
    assert len(feats) == len(want)
    for f, (h, vals) in zip(feats, want):
        for i, v in enumerate(vals):
            assert f[i] == pytest.approx(float(v), rel=1e-5, abs=1e-7), f"ef {ef} k {k} hop {h} f{i}"


def _check_search(ix, O, q, k, ef, **kw):
    qd = torch.from_numpy(q).cuda()
    ids, dists, st = ix.search(qd, k, ef, stats=True, **{a: b for a, b in kw.items() if a != "mlp_np"})
    ids, dists, st = _np(ids).view(np.uint32), _np(dists), _np(st)
    okw = dict(eps0=kw.get("eps0", 0.0), multi_estimate=kw.get("multi_estimate", True))
    if kw.get("hop_cap"):
        okw["hop_cap"] = kw["hop_cap"]
    if kw.get("mlp_np") is not None:
        okw.update(mlp=kw["mlp_np"], stop_logit=kw.get("stop_logit", 0.0), stop_every=kw.get("stop_every", 1))
    for i in range(q.shape[0]):
        oi, od, oh, os_ = O.search(q[i], k, ef, **okw)
        np.testing.assert_array_equal(ids[i], oi, err_msg=f"query {i} ids")
        np.testing.assert_array_equal(dists[i], od, err_msg=f"query {i} dists")
        assert (st[i, 0], st[i, 1]) == (oh, os_), f"query {i}: hops/status {st[i]} vs {(oh, os_)}"
    return ids, dists, st


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("ef", [10, 16, 33, 64, 128, 300])
def test_search_parity_r32(gpu_tiny, oracle_mod, ef, kernel):
    """Algorithm 1 with multiple estimates and implicit re-ranking: ids,
    distances and hop counts identical to the oracle (kernel 0: the compact
    kernel up to ef 64; 1: the general kernel throughout)."""
    ix, p, x, q = gpu_tiny
    _check_search(ix, oracle_mod.Index(p), q, 10, ef, kernel=kernel)


@pytest.mark.parametrize("kernel", [0, 1])
@pytest.mark.parametrize("ef", [16, 64, 100, 200])
def test_search_parity_r64(gpu_tiny64, oracle_mod, ef, kernel):
    """Out-degree 64 (two neighbours per lane); kernel 0 takes the compact
    kernel up to ef 128, 1 the general kernel."""
    ix, p, x, q = gpu_tiny64
    _check_search(ix, oracle_mod.Index(p), q, 10, ef, kernel=kernel)


def test_search_variants(gpu_tiny, oracle_mod):
    """eps0 admission key, the w/o-ME ablation and a binding hop cap."""
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    _check_search(ix, O, q, 10, 64, eps0=1.0)
    _check_search(ix, O, q, 10, 64, multi_estimate=False)
    _, _, st = _check_search(ix, O, q, 5, 64, hop_cap=7)
    assert np.all(st[:, 0] <= 7) and np.any(st[:, 1] == 1)


def test_search_k_equals_ef_and_k1(gpu_tiny, oracle_mod):
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    _check_search(ix, O, q, 1, 1)
    _check_search(ix, O, q, 1, 40)
    _check_search(ix, O, q, 100, 100)
    _check_search(ix, O, q, 256, 256)


def test_mixed_k_ef_ragged_batch(gpu_tiny, oracle_mod):
    """One launch with per-query k and ef (the persistent work queue):
    each query's slice of the ragged output equals the oracle's search."""
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    rng = np.random.default_rng(3)
    nq = q.shape[0]
    k = rng.choice([1, 10, 100], size=nq).astype(np.int32)
    ef = np.array([rng.integers(kk, 8 * kk + 1) for kk in k], dtype=np.int32)
    ids, dists, st = ix.search(torch.from_numpy(q).cuda(), torch.from_numpy(k), torch.from_numpy(ef), stats=True)
    ids, dists, st = _np(ids).view(np.uint32), _np(dists), _np(st)
    off = np.concatenate([[0], np.cumsum(k)])
    assert ids.shape[0] == off[-1]
    for i in range(nq):
        oi, od, oh, os_ = O.search(q[i], int(k[i]), int(ef[i]))
        np.testing.assert_array_equal(ids[off[i]:off[i + 1]], oi)
        np.testing.assert_array_equal(dists[off[i]:off[i + 1]], od)
        assert st[i, 0] == oh


@pytest.mark.parametrize("kernel", [1, 2])
def test_uniform_k_outputs_without_planning(gpu_tiny, oracle_mod, kernel):
    """uniform_k: outputs at i * k with no prefix sum.  Identical to the
    ragged launch of the same k[]; a query whose k differs is padding with
    SQG_STATUS_BAD_PARAM and the rest are untouched; max_k other than
    uniform_k is rejected."""
    from paper_2411_12229_gb300 import _binding as B
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    nq, k, ef = q.shape[0], 10, 40
    qd = torch.from_numpy(q).cuda()
    kt = torch.full((nq,), k, dtype=torch.int32)
    et = torch.full((nq,), ef, dtype=torch.int32)
    r_ids, r_d, r_st = ix.search(qd, kt, et, stats=True, kernel=kernel, max_k=k, max_ef=ef)
    u_ids, u_d, u_st = ix.search(qd, kt, et, stats=True, kernel=kernel, max_k=k, max_ef=ef, uniform_k=k)
    assert torch.equal(r_ids, u_ids.flatten()) and torch.equal(r_d, u_d.flatten()) and torch.equal(r_st, u_st)
    s_ids, s_d = ix.search(qd, k, ef, kernel=kernel)  # scalar k takes this path by itself
    assert torch.equal(s_ids, u_ids) and torch.equal(s_d, u_d)
    kt[3], kt[7] = 5, 11
    m_ids, m_d, m_st = ix.search(qd, kt, et, stats=True, kernel=kernel, max_k=k, max_ef=ef, uniform_k=k)
    m_ids, m_d, m_st = _np(m_ids).view(np.uint32).reshape(nq, k), _np(m_d).reshape(nq, k), _np(m_st)
    for i in range(nq):
        if i in (3, 7):
            assert m_st[i, 1] == B.STATUS_BAD_PARAM and np.all(m_ids[i] == 0xFFFFFFFF) and np.all(np.isinf(m_d[i]))
        else:
            oi, od, oh, _ = O.search(q[i], k, ef)
            np.testing.assert_array_equal(m_ids[i], oi)
            np.testing.assert_array_equal(m_d[i], od)
            assert m_st[i, 0] == oh
    assert ix.status() & B.STATUS_BAD_PARAM
    with pytest.raises(RuntimeError):
        ix.search(qd, kt, et, max_k=12, max_ef=ef, uniform_k=k)


def test_plain_sqg_search_entry_point(gpu_tiny, oracle_mod):
    """sqg_search (device k[], ef[], bounds read on the device)."""
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    nq = q.shape[0]
    k = torch.full((nq,), 10, dtype=torch.int32, device="cuda")
    ef = torch.full((nq,), 48, dtype=torch.int32, device="cuda")
    ids = torch.empty(nq * 10, dtype=torch.int32, device="cuda")
    dd = torch.empty(nq * 10, dtype=torch.float32, device="cuda")
    ix.search_plain(torch.from_numpy(q).cuda(), k, ef, ids, dd)
    ids = _np(ids).view(np.uint32).reshape(nq, 10)
    for i in range(nq):
        np.testing.assert_array_equal(ids[i], O.search(q[i], 10, 48)[0])


def test_invalid_per_query_params_are_padding(gpu_tiny, oracle_mod):
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    k = np.array([10, 0, 10, 5, 300, 10], dtype=np.int32)
    ef = np.array([32, 32, 5, 5, 400, 40], dtype=np.int32)
    qq = torch.from_numpy(q[:6]).cuda()
    ids, dists, st = ix.search(qq, torch.from_numpy(k), torch.from_numpy(ef), stats=True, max_k=10, max_ef=40)
    ids, dists, st = _np(ids).view(np.uint32), _np(dists), _np(st)
    kk = np.clip(k, 0, 256)
    off = np.concatenate([[0], np.cumsum(kk)])
    assert ids.shape[0] == off[-1]
    bad = [1, 2, 4]
    for i in range(6):
        sl = slice(off[i], off[i + 1])
        if i in bad:
            assert st[i, 1] == 4 and np.all(ids[sl] == 0xFFFFFFFF) and np.all(np.isinf(dists[sl]))
        else:
            np.testing.assert_array_equal(ids[sl], O.search(q[i], int(k[i]), int(ef[i]))[0])
    assert ix.status() & 4
    assert ix.status() == 0  # cleared by the read


def test_empty_batch_and_bad_arguments(gpu_tiny):
    from paper_2411_12229_gb300._binding import SqgError
    ix, p, x, q = gpu_tiny
    ids, dists = ix.search(torch.empty((0, ix.d), device="cuda"), 10, 32)
    assert ids.numel() == 0
    with pytest.raises(SqgError):
        ix.search(torch.from_numpy(q).cuda(), 10, 32, hop_cap=-1)
    with pytest.raises(SqgError):
        ix.search(torch.from_numpy(q).cuda(), 10, 32, max_k=300)
    with pytest.raises(SqgError):  # workspace too small
        ix.search(torch.from_numpy(q).cuda(), 10, 32, max_k=10, max_ef=32,
                  workspace=torch.empty(16, dtype=torch.uint8, device="cuda"))


def test_caller_workspace_matches_own_allocation(gpu_tiny):
    ix, p, x, q = gpu_tiny
    qd = torch.from_numpy(q).cuda()
    a = ix.search(qd, 10, 64)
    nbytes = ix.workspace_size(q.shape[0], 10, 64)
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    b = ix.search(qd, 10, 64, max_k=10, max_ef=64, workspace=ws)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


@pytest.mark.parametrize("ef,smem_log2", [(64, 5), (300, 6), (1024, 0)])
def test_visited_set_migration(gpu_tiny, oracle_mod, ef, smem_log2):
    """A search whose expansions fill half of the shared-memory visited table
    continues in the warp's full-size table in the workspace; the search is
    unchanged (32- and 64-slot tables force the move on this index)."""
    ix, p, x, q = gpu_tiny
    _, _, st = _check_search(ix, oracle_mod.Index(p), q, 10, ef, visited_smem_log2=smem_log2)
    if smem_log2:
        assert st[:, 0].min() > (1 << smem_log2) // 2


def test_speculative_prefetch_changes_nothing(gpu_tiny, oracle_mod):
    ix, p, x, q = gpu_tiny
    _check_search(ix, oracle_mod.Index(p), q, 10, 64, prefetch=2)
    _check_search(ix, oracle_mod.Index(p), q, 10, 64, prefetch=2, warps_per_block=1)


@pytest.mark.parametrize("kernel", [1, 2])
def test_learned_stop_constant_networks(gpu_tiny, oracle_mod, kernel):
    """kernel 1: the stop fused into the general kernel; 2: into the
    compact kernel's stop build."""
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    mlp = np.zeros(5313, np.float32)
    for b3, want in ((-100.0, 0), (100.0, 2)):
        mlp[-1] = b3
        dm = torch.from_numpy(mlp).cuda()
        _, _, st = _check_search(ix, O, q, 10, 64, stop_mlp=dm, mlp_np=mlp, stop_logit=0.0, stop_every=4,
                                 kernel=kernel)
        assert np.all(st[:, 1] == want)


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("ef", [64, 100])
def test_learned_stop_random_network_parity(gpu_tiny, oracle_mod, kernel, ef):
    """A random network: the fused fp32 forward takes the same stop decision
    at the same hop as the oracle's forward (both kernels; 2 and 4 beam
    slots per lane in the compact one)."""
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    rng = np.random.default_rng(5)
    mlp = (rng.standard_normal(5313) * 0.3).astype(np.float32)
    dm = torch.from_numpy(mlp).cuda()
    for thr in (-1.0, 0.5, 2.0):
        _check_search(ix, O, q, 10, ef, stop_mlp=dm, mlp_np=mlp, stop_logit=thr, stop_every=2, kernel=kernel)


@pytest.mark.parametrize("kernel", [1, 2])
def test_learned_stop_edges(gpu_tiny, gpu_tiny64, oracle_mod, kernel):
    """The stop with a binding hop cap, the error-bound key, every hop
    (the last expansion of a search that ends by itself included), small k
    and out-degree 64 (two neighbours per lane)."""
    rng = np.random.default_rng(8)
    mlp = (rng.standard_normal(5313) * 0.3).astype(np.float32)
    dm = torch.from_numpy(mlp).cuda()
    kw = dict(stop_mlp=dm, mlp_np=mlp, kernel=kernel)
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    _check_search(ix, O, q, 10, 64, stop_logit=1.0, stop_every=3, hop_cap=20, **kw)
    _check_search(ix, O, q, 10, 48, stop_logit=1.0, stop_every=2, eps0=1.9, **kw)
    _, _, st = _check_search(ix, O, q, 1, 8, stop_logit=3.0, stop_every=1, **kw)
    ix, p, x, q = gpu_tiny64
    O = oracle_mod.Index(p)
    for ef in (40, 128):
        _check_search(ix, O, q, 10, ef, stop_logit=0.5, stop_every=2, **kw)


def test_trace_features_bit_exact(gpu_tiny, oracle_mod):
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    nq = 24
    gt = np.stack([oracle_mod.bruteforce(x, q[i], 10)[0] for i in range(nq)]).astype(np.int32)
    ids, dists, st, feats, hits, cnt = ix.search_trace(torch.from_numpy(q[:nq]).cuda(), 10, 64,
                                                       torch.from_numpy(gt).cuda(), 256, stop_every=3)
    feats, hits, cnt = _np(feats), _np(hits), _np(cnt)
    for i in range(nq):
        r = O.search(q[i], 10, 64, stop_every=3, gt=gt[i].view(np.uint32), trace_cap=256)
        tf, th = r[4], r[5]
        assert cnt[i] == len(tf)
        np.testing.assert_array_equal(feats[i, :cnt[i]], tf)
        np.testing.assert_array_equal(hits[i, :cnt[i]], th)


@pytest.fixture(scope="module")
def shaped_index(shaped_index_file):
    from paper_2411_12229_gb300.api import Index
    p, x, q = shaped_index_file
    return Index(p, 0), p, x, q


def test_other_shapes_parity(shaped_index, oracle_mod):
    """The kernel instantiations for d = 96 (24 of 32 lanes hold the raw
    vector), 256, 960 (R = 64) and 1536: prepared queries, estimates and
    searches identical to the oracle."""
    ix, p, x, q = shaped_index
    O = oracle_mod.Index(p)
    qd = torch.from_numpy(q).cuda()
    qrot, planes, scal = ix.prepare_queries(qd)
    qrot = _np(qrot)
    for i in range(0, q.shape[0], 5):
        np.testing.assert_array_equal(qrot[i], O.prepare_query(q[i])["qrot"])
    v = (np.arange(q.shape[0]) * 37 % ix.n).astype(np.int32)
    S, est, key, dc = (_np(t) for t in ix.estimate_block(qd, torch.from_numpy(v), 1.0))
    for i in range(0, q.shape[0], 3):
        r = O.estimate_block(q[i], int(v[i]), 1.0)
        np.testing.assert_array_equal(S[i], r["S"])
        np.testing.assert_array_equal(est[i], r["est"])
        np.testing.assert_array_equal(key[i], r["key"])
    for ef in (10, 40, 100):
        _check_search(ix, O, q, 10, ef)
    if ix.d <= 1024:  # the compact kernel's range: its output is the general kernel's
        big = ((100, 160), (10, 256)) if ix.d <= 256 else ()  # k <= 128 and ef <= 256 for d <= 256
        for k, ef in ((10, 40), (10, 128)) + big:
            c = ix.search(qd, k, ef, stats=True, kernel=2)
            g = ix.search(qd, k, ef, stats=True, kernel=1)
            assert all(torch.equal(u, v) for u, v in zip(c, g))
        for k, ef in big:
            _check_search(ix, O, q[:16], k, ef, kernel=2)


def test_other_shapes_learned_stop(shaped_index, oracle_mod):
    """The fused stop with a random network on the other workloads' shapes:
    the compact kernel's stop builds for d = 96 and 256 (features through
    shared memory) and for d = 960 at out-degree 64 (features in
    registers), beams of 2 and 4 slots per lane, and the general kernel at
    every shape (d = 1536 included): stop decisions, hops, ids and
    distances identical to the oracle's."""
    ix, p, x, q = shaped_index
    O = oracle_mod.Index(p)
    rng = np.random.default_rng(17)
    mlp = (rng.standard_normal(5313) * 0.3).astype(np.float32)
    dm = torch.from_numpy(mlp).cuda()
    q = q[:24]
    stopped = 0
    for kernel in ((1, 2) if ix.d <= 1024 else (1,)):
        for ef, every, thr in ((40, 3, -1.0), (100, 2, 1.5)):
            _, _, st = _check_search(ix, O, q, 10, ef, stop_mlp=dm, mlp_np=mlp, stop_logit=thr, stop_every=every,
                                     kernel=kernel)
            stopped += int(np.count_nonzero(st[:, 1] & 2))  # SQG_STATUS_LEARNED_STOP
    assert stopped > 0  # the network's decision was exercised


@pytest.mark.parametrize("ef", [16, 64])
def test_expansion_order_identical(gpu_tiny, oracle_mod, ef):
    """Algorithm 1 line 3: the sequence of expanded vertices, hop by hop,
    is the oracle's (the strongest form of search-path parity)."""
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    r = ix.search_trace(torch.from_numpy(q).cuda(), 10, ef, None, 0, path_cap=512)
    st, path = _np(r[2]), _np(r[-1]).view(np.uint32)
    for i in range(q.shape[0]):
        opath = O.search(q[i], 10, ef, path_cap=512)[-1]
        assert st[i, 0] == len(opath)
        np.testing.assert_array_equal(path[i, :len(opath)], opath)
        assert np.all(path[i, len(opath):] == 0xFFFFFFFF)


def test_device_payload_corruption_is_rejected(tiny_index, tmp_path):
    import pathlib

    from paper_2411_12229_gb300._binding import SqgError
    from paper_2411_12229_gb300.api import Index
    data = bytearray(pathlib.Path(tiny_index[0]).read_bytes())
    data[-200] ^= 1
    bad = tmp_path / "bad.sqg"
    bad.write_bytes(bytes(data))
    with pytest.raises(SqgError) as e:
        Index(bad, 0)
    assert e.value.code == -3


def test_host_buffers_end_to_end(gpu_tiny, oracle_mod):
    ix, p, x, q = gpu_tiny
    ids, dists = ix.search_host(q, 10, 64)
    O = oracle_mod.Index(p)
    for i in range(0, q.shape[0], 7):
        np.testing.assert_array_equal(ids[i].view(np.uint32), O.search(q[i], 10, 64)[0])


def test_max_k_and_max_ef(gpu_tiny, oracle_mod):
    """k = SQG_MAX_K (256) and ef = SQG_MAX_EF (2048) on the 2,000-vertex
    graph: the largest result and beam the kernels take.  With multiple
    estimates the beam fills with copies (visited copies keep their slots,
    R5) long before the graph is exhausted; both sides stop at the same
    hop, past the visited set's move to global memory (128 shared slots
    here, moved at 64 expansions)."""
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    ids, dists, st = _check_search(ix, O, q[:16], 256, 2048, visited_smem_log2=7)
    assert np.all(st[:, 1] == 0) and np.all(st[:, 0] > 64)


@pytest.fixture(scope="module")
def gpu_ties(tmp_path_factory, lib_built):
    """Integer-valued vectors, a fifth of them exact copies of others: many
    equal distances and keys (ordered by id, R4) and neighbours equal to
    their centre (zero codes and factors, R3); queries with integer values
    and some equal to data vectors (distance 0)."""
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300.api import Index
    rng = np.random.default_rng(42)
    base = rng.integers(-2, 3, size=(1200, 64)).astype(np.float32)
    x = np.concatenate([base, base[rng.integers(0, 1200, 300)]])
    x = x[rng.permutation(x.shape[0])]
    q = rng.integers(-2, 3, size=(48, 64)).astype(np.float32)
    q[:8] = x[rng.integers(0, x.shape[0], 8)]
    p = tmp_path_factory.mktemp("ties") / "ties.sqg"
    ib.build_index(p, x, 32)
    return Index(p, 0), p, x, q


def test_ties_and_duplicates_parity(gpu_ties, oracle_mod):
    ix, p, x, q = gpu_ties
    O = oracle_mod.Index(p)
    for ef in (16, 64, 200):
        ids, dists, st = _check_search(ix, O, q, 10, ef)
    assert np.all(dists[:8, 0] == 0.0)  # the query's own vector
    _check_search(ix, O, q, 10, 64, eps0=1.9)
    _check_search(ix, O, q, 10, 64, multi_estimate=False)


def test_bounded_wait_runs_out_and_the_context_stays_usable(gpu_tiny, oracle_mod):
    """Failure detection without a GPU fault: the search kernel's bounded
    wait, on an mbarrier phase that nothing completes, gives up after its
    1 s limit and reports SQG_STATUS_TIMEOUT; searches still run after it."""
    import ctypes as C

    from paper_2411_12229_gb300 import _binding as B
    status, ns = C.c_uint32(0), C.c_uint64(0)
    assert B.lib().sqg_wait_selftest(0, C.byref(status), C.byref(ns)) == 0
    assert status.value == 8  # SQG_STATUS_TIMEOUT
    assert 1.0e9 <= ns.value < 10.0e9
    ix, p, x, q = gpu_tiny
    _check_search(ix, oracle_mod.Index(p), q[:8], 10, 32)


def test_more_results_than_vertices_are_padded_on_the_gpu(lib_built, oracle_mod, tmp_path):
    """k = 100 on a 60-vertex graph: the 60 vertices, then padding, as the
    oracle gives them (ids, distances, hops)."""
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300.api import Index
    rng = np.random.default_rng(61)
    x = rng.standard_normal((60, 32)).astype(np.float32)
    p = tmp_path / "n60.sqg"
    ib.build_index(p, x, 32)
    ix = Index(p, 0)
    q = rng.standard_normal((7, 32)).astype(np.float32)
    ids, dists, st = _check_search(ix, oracle_mod.Index(p), q, 100, 300)
    assert np.all(ids[:, 60:] == 0xFFFFFFFF) and np.all(np.isinf(dists[:, 60:]))

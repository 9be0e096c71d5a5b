"""Host-side tests (no GPU): the C ABI's exports and host error paths, the
index builder against the oracle's definitions, and the input generators."""

import ctypes as C
import pathlib
import re

import numpy as np
import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]


def header_functions():
    text = (ROOT / "include" / "sqg.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sqg_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(lib_built):
    from paper_2411_12229_gb300 import _binding
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib_built, n), f"libsqg.so does not export {n}"
    assert set(names) == set(_binding.exported_symbols())


def test_error_strings(lib_built):
    for code in range(0, -9, -1):
        s = lib_built.sqg_error_string(code)
        assert s and s != b"unknown error"
    assert lib_built.sqg_error_string(-99) == b"unknown error"


def test_index_load_host_errors(lib_built, tmp_path, tiny_index):
    h = C.c_void_p()
    assert lib_built.sqg_index_load(str(tmp_path / "missing.sqg").encode(), 0, C.byref(h)) == -2
    junk = tmp_path / "junk.sqg"
    junk.write_bytes(b"NOPE" * 100)
    assert lib_built.sqg_index_load(str(junk).encode(), 0, C.byref(h)) == -3
    data = pathlib.Path(tiny_index[0]).read_bytes()
    trunc = tmp_path / "trunc.sqg"
    trunc.write_bytes(data[: len(data) - 128])
    assert lib_built.sqg_index_load(str(trunc).encode(), 0, C.byref(h)) == -3
    bad_hdr = bytearray(data[:4096])
    bad_hdr[16] ^= 1  # d
    hdr = tmp_path / "hdr.sqg"
    hdr.write_bytes(bytes(bad_hdr) + data[4096:])
    assert lib_built.sqg_index_load(str(hdr).encode(), 0, C.byref(h)) == -3
    assert lib_built.sqg_index_load(None, 0, C.byref(h)) == -1
    assert lib_built.sqg_index_load(str(tiny_index[0]).encode(), -1, C.byref(h)) == -1


def test_oracle_rejects_corrupt_payload(oracle_mod, tiny_index, tmp_path):
    data = bytearray(pathlib.Path(tiny_index[0]).read_bytes())
    data[len(data) // 2] ^= 0x40
    p = tmp_path / "flip.sqg"
    p.write_bytes(bytes(data))
    with pytest.raises(OSError):
        oracle_mod.Index(p)


def test_builder_codes_and_factors_match_the_definition(oracle_mod, tiny_index):
    """The file's codes and factors (written by the library's host builder)
    against the oracle's fp64 RaBitQ quantization of each edge (Eq. (3) with
    the vertex as centre, Sec. 3.1.1)."""
    p, x, _ = tiny_index
    O = oracle_mod.Index(p)
    rot = O.rotation()
    rng = np.random.default_rng(0)
    flips = 0
    for v in rng.choice(O.n, 25, replace=False):
        blk = O.vertex(int(v))
        np.testing.assert_array_equal(O.raw(int(v)), x[v])
        for j in range(O.R):
            o = int(blk["ids"][j])
            bits, f = oracle_mod.quantize_edge(rot, x[v], x[o])
            vrot = rot.astype(np.float64) @ (x[o].astype(np.float64) - x[v]) / f["n_o"]
            diff = bits != blk["bits"][j]
            assert np.all(np.abs(vrot[diff]) < 1e-5), "a code bit differs away from a sign tie"
            flips += int(diff.sum())
            assert blk["popcount"][j] == blk["bits"][j].sum()
            for name in ("f_add", "f_rescale", "f_err"):
                assert blk[name][j] == pytest.approx(f[name], rel=2e-5, abs=2e-5 * abs(f["f_add"]))
    assert flips <= 2


def test_graph_invariants(oracle_mod, tiny_index):
    """Every vertex has exactly R distinct out-neighbours, no self loop
    (Sec. 3.2.2, degree aligned to the batch of 32), and every vertex is
    reachable from the entry point."""
    p, x, _ = tiny_index
    O = oracle_mod.Index(p)
    adj = np.stack([O.vertex(v)["ids"] for v in range(O.n)])
    assert adj.shape == (O.n, 32)
    assert np.all(adj < O.n)
    assert np.all(adj != np.arange(O.n)[:, None])
    s = np.sort(adj, axis=1)
    assert np.all(s[:, 1:] != s[:, :-1])
    seen = np.zeros(O.n, bool)
    stack = [O.entry]
    seen[O.entry] = True
    while stack:
        u = stack.pop()
        for v in adj[u]:
            if not seen[v]:
                seen[v] = True
                stack.append(v)
    assert seen.all()


def test_entry_is_the_medoid(oracle_mod, tiny_index):
    p, x, _ = tiny_index
    O = oracle_mod.Index(p)
    mean = x.astype(np.float64).mean(axis=0)
    d = np.sum((x - mean) ** 2, axis=1)
    assert O.entry == int(np.argmin(d))


def test_block_size_formula(oracle_mod, tiny_index, tiny_index_r64):
    """Sec. 3.3: n(32D + 32R + DR) bits for vectors, ids and codes; the
    block adds 3 fp32 factors and a popcount per neighbour, padded to 128 B."""
    for p, R in ((tiny_index[0], 32), (tiny_index_r64[0], 64)):
        O = oracle_mod.Index(p)
        bits = 32 * O.d + 32 * R + O.d * R
        assert O.block_bytes == -(-(bits // 8 + 16 * R) // 128) * 128
    assert (4 * 128 + 4 * 32 + 128 * 32 // 8 + 16 * 32) == 1664  # d=128, R=32
    assert (4 * 960 + 4 * 64 + 960 * 64 // 8 + 16 * 64) == 12800  # d=960, R=64


def test_knn_host_matches_bruteforce(lib_built, oracle_mod):
    from paper_2411_12229_gb300 import index_builder as ib
    rng = np.random.default_rng(1)
    x = rng.standard_normal((300, 64)).astype(np.float32)
    nn = ib.knn_host(x, 8)
    for i in range(0, 300, 37):
        ids, _ = oracle_mod.bruteforce(x, x[i], 9)
        assert ids[0] == i
        np.testing.assert_array_equal(nn[i], ids[1:])


def test_random_rotation_is_orthogonal():
    from paper_2411_12229_gb300 import index_builder as ib
    for d in (32, 128, 960):
        R = ib.random_rotation(d, 2).astype(np.float64)
        assert np.abs(R @ R.T - np.eye(d)).max() < 1e-5


def test_random_graph_is_simple():
    from paper_2411_12229_gb300 import index_builder as ib
    adj = ib.random_graph(500, 32, 3)
    assert np.all(adj != np.arange(500)[:, None])
    s = np.sort(adj, axis=1)
    assert np.all(s[:, 1:] != s[:, :-1])


def test_synth_is_deterministic_and_chunk_independent():
    from paper_2411_12229_gb300 import synth
    w = synth.Workload("t", 70_000, 32, 16, 10, 32, dim_scale="loguniform")
    full = synth.base(w)
    np.testing.assert_array_equal(full[65_000:66_000], synth.base(w, 65_000, 66_000))
    np.testing.assert_array_equal(synth.queries(w), synth.queries(w))
    assert not np.array_equal(synth.queries(w)[0], full[0])


def test_workload_recipes():
    from paper_2411_12229_gb300 import synth
    W = synth.WORKLOADS
    t = W["tiny-10k-d128"]
    assert (t.n, t.d, t.n_components, t.n_queries, t.degree, t.k, t.ef) == (10_000, 128, 64, 200, 32, 10,
                                                                               (32, 64, 128))
    b = W["batched-1m-d128"]
    assert (b.n, b.d, b.n_components, b.n_queries, b.degree, b.dim_scale) == (1_000_000, 128, 1024, 10_000, 32,
                                                                              "loguniform")
    assert min(b.ef) == 16 and max(b.ef) == 512
    h = W["highdim-1m-d960"]
    assert (h.n, h.d, h.degree, h.n_train, h.dim_scale) == (1_000_000, 960, 64, 50_000, "power")
    u = W["uneven-1m-d1536"]
    assert (u.n, u.d, u.degree, u.n_queries, u.unit_norm, u.mixed_k) == (1_000_000, 1536, 32, 20_000, True,
                                                                         (1, 10, 100))
    s = W["serving-4m-d96"]
    assert (s.n, s.d, s.n_components, s.degree) == (4_000_000, 96, 4096, 32)
    # value distributions
    hs = synth.small(h, 2000, 10)
    xh = synth.base(hs)
    assert xh.min() >= 0
    v = xh.var(axis=0)
    assert v[:10].mean() > v[-100:].mean()
    xu = synth.base(synth.small(u, 500, 10))
    np.testing.assert_allclose(np.linalg.norm(xu, axis=1), 1.0, rtol=1e-5)
    k, ef = synth.query_k_ef(u, 1000)
    assert set(np.unique(k)) == {1, 10, 100} and np.all(ef >= k) and np.all(ef <= 8 * k)
    arr = synth.poisson_arrivals(1000.0, 5000)
    assert np.all(np.diff(arr) > 0) and abs(5000 / arr[-1] - 1000) < 100


def test_fjlt_builder_agrees_with_the_oracle(oracle_mod, lib_built):
    """Two implementations of the same definitions: the builder's signs and
    dense fast-JLT matrix against the oracle's generator and transform."""
    from paper_2411_12229_gb300 import index_builder as ib
    for d in (32, 128, 256):
        s = ib.fjlt_signs(d, 11)
        np.testing.assert_array_equal(s, oracle_mod.fjlt_signs(11, d))
        M = ib.fjlt_matrix(d, 11).astype(np.float64)
        rng = np.random.default_rng(d)
        x = rng.standard_normal(d).astype(np.float32)
        np.testing.assert_allclose(M @ x.astype(np.float64), oracle_mod.fjlt_f64(s, x), rtol=0, atol=1e-5)
    with pytest.raises(ValueError):
        ib.fjlt_matrix(96, 1)


def test_fjlt_index_header_and_writer_checks(lib_built, oracle_mod, tmp_path):
    """The fast-JLT writer refuses a d that is not a power of 2 or an
    unknown rotation kind; a written index carries format version 2 and
    loads in the oracle with the generator's signs."""
    from paper_2411_12229_gb300 import _binding as B
    from paper_2411_12229_gb300 import index_builder as ib
    rng = np.random.default_rng(0)
    x = rng.standard_normal((100, 96)).astype(np.float32)
    adj = ib.random_graph(100, 32, 1)
    rot = np.eye(96, dtype=np.float32)
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    for kind in (1, 2):
        rc = B.lib().sqg_write_index2(str(tmp_path / "bad.sqg").encode(), ptr(x), 100, 96, ptr(adj), 32, ptr(rot),
                                      0, 5, 3, 1, kind, 0)
        assert rc == -1  # SQG_ERR_INVALID_ARG
    p = tmp_path / "ok.sqg"
    ib.build_index(p, x, 32, rotation="fjlt")
    with open(p, "rb") as f:
        assert int.from_bytes(f.read(8)[4:8], "little") == 2
    O = oracle_mod.Index(p)
    assert O.d == 128
    np.testing.assert_array_equal(O.fjlt_signs(), ib.fjlt_signs(128, 2))


def _rehash_header(buf: bytearray) -> None:
    """FNV-1a 64 over the header's first twelve little-endian u64 words."""
    h = 0xCBF29CE484222325
    for i in range(0, 96, 8):
        h = ((h ^ int.from_bytes(buf[i:i + 8], "little")) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    buf[96:104] = h.to_bytes(8, "little")


def test_metric_field_and_writer_checks(lib_built, oracle_mod, tiny_index, tmp_path):
    """Metric 0 (squared Euclidean) and 1 (cosine) load; any other value is
    a format error for the library and the oracle.  The writer takes metric
    1 only for unit (or zero) vectors; the builder normalizes the data."""
    from paper_2411_12229_gb300 import _binding as B
    from paper_2411_12229_gb300 import index_builder as ib
    data = bytearray(pathlib.Path(tiny_index[0]).read_bytes())
    h = C.c_void_p()
    for metric, ok in ((0, True), (1, True), (2, False), (7, False)):
        buf = bytearray(data)
        buf[32:36] = metric.to_bytes(4, "little")
        _rehash_header(buf)
        p = tmp_path / f"m{metric}.sqg"
        p.write_bytes(bytes(buf))
        if ok:
            assert oracle_mod.Index(p).metric == metric
        else:
            assert lib_built.sqg_index_load(str(p).encode(), 0, C.byref(h)) == -3
            with pytest.raises(OSError):
                oracle_mod.Index(p)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((100, 64)).astype(np.float32)
    adj = ib.random_graph(100, 32, 1)
    rot = np.eye(64, dtype=np.float32)
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    out = str(tmp_path / "w.sqg").encode()
    assert B.lib().sqg_write_index2(out, ptr(x), 100, 64, ptr(adj), 32, ptr(rot), 0, 5, 3, 1, 0, 1) == -1
    assert B.lib().sqg_write_index2(out, ptr(x), 100, 64, ptr(adj), 32, ptr(rot), 0, 5, 3, 1, 0, 2) == -1
    xu = ib.unit_rows(x)
    xu[7] = 0.0  # a zero vector is allowed
    assert B.lib().sqg_write_index2(out, ptr(xu), 100, 64, ptr(adj), 32, ptr(rot), 0, 5, 3, 1, 0, 1) == 0
    assert oracle_mod.Index(tmp_path / "w.sqg").metric == 1
    np.testing.assert_allclose(np.linalg.norm(np.delete(xu, 7, 0).astype(np.float64), axis=1), 1.0, atol=1e-6)
    with pytest.raises(ValueError):
        ib.build_index(tmp_path / "b.sqg", x, 32, metric="dot")
    ib.build_index(tmp_path / "c.sqg", x, 32, metric="cosine")
    O = oracle_mod.Index(tmp_path / "c.sqg")
    assert O.metric == 1
    np.testing.assert_allclose(O.raw_all(), ib.unit_rows(x), rtol=0, atol=0)


@pytest.mark.parametrize("n,d,R,L", [(600, 64, 32, 64), (400, 160, 32, 96)])
def test_host_graph_adjust_matches_the_oracle(oracle_mod, lib_built, n, d, R, L):
    """The builder's prune, reverse edges, re-prune and angle rule give the
    oracle's lists exactly (same distance order, same (dist, id) order)
    when no list needs the random fill and no reachability repair ran."""
    from paper_2411_12229_gb300 import index_builder as ib
    rng = np.random.default_rng(n)
    cen = rng.standard_normal((8, d)) * 3
    x = (cen[rng.integers(0, 8, n)] + rng.standard_normal((n, d))).astype(np.float32)
    dist = ((x[:, None, :].astype(np.float64) - x[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(dist, np.inf)
    cand = np.argsort(dist, axis=1, kind="stable")[:, :L].astype(np.uint32)
    cand[::7, -3:] = rng.integers(0, n, (cand[::7].shape[0], 3))  # some repeats and far ids
    cand[::11, 1] = np.arange(0, n, 11)  # self ids, dropped
    adj, st = ib.build_graph(x, cand, R, 0, 3, 0)
    assert st["random_filled"] == 0 and st["repairs"] == 0
    out, cnt = oracle_mod.adjust_graph(x, cand, R)
    assert np.all(cnt == R)
    np.testing.assert_array_equal(adj, out)


def test_builder_needs_more_vectors_than_the_degree(lib_built, tmp_path):
    """The loader takes only R distinct neighbours per vertex, none itself,
    so an index of degree R needs n > R vectors."""
    from paper_2411_12229_gb300 import index_builder as ib
    x = np.random.default_rng(0).standard_normal((32, 32)).astype(np.float32)
    with pytest.raises(ValueError):
        ib.build_index(tmp_path / "t.sqg", x, 32)
    ib.build_index(tmp_path / "ok.sqg", np.vstack([x, x[:1] + 1]), 32)


def test_host_irregular_graph_matches_the_oracle(oracle_mod, lib_built):
    """The degree-unaligned build ("w/o GR"): the host rows are the oracle's
    lists without the angle rule, empty slots NO_ID."""
    from paper_2411_12229_gb300 import index_builder as ib
    rng = np.random.default_rng(7)
    n, d, R = 500, 64, 32
    cen = rng.standard_normal((8, d)) * 3
    x = (cen[rng.integers(0, 8, n)] + rng.standard_normal((n, d))).astype(np.float32)
    dist = ((x[:, None, :].astype(np.float64) - x[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(dist, np.inf)
    cand = np.argsort(dist, axis=1, kind="stable")[:, :64].astype(np.uint32)
    adj, st = ib.build_graph(x, cand, R, 0, 3, 0, regular=False)
    assert st["supplemented"] == 0 and st["random_filled"] == 0
    if st["repairs"] == 0:
        out, cnt = oracle_mod.adjust_graph(x, cand, R, regular=False)
        np.testing.assert_array_equal(adj, out)
    assert np.any(adj == 0xFFFFFFFF)


def test_recall_and_distance_ratio_on_hand_made_cases():
    """Sec. 5.1's accuracy metrics: recall |G cap S| / K per query, averaged
    (padding ids -1 never count), and the average distance ratio over ranks
    of ||o_i - q|| / ||o*_i - q|| from squared distances (ranks whose true
    distance is 0 skipped, unreachable results skipped)."""
    from paper_2411_12229_gb300 import eval as E
    gt = np.array([[1, 2, 3, 4], [5, 6, 7, 8]])
    ids = np.array([[4, 3, 9, -1], [5, 6, 7, 8]])
    assert E.recall(ids, gt, 4) == 0.75  # 2/4 and 4/4
    assert E.recall(ids, gt, 2) == 0.5  # {4, 3} vs {1, 2}: 0; {5, 6}: 2
    np.testing.assert_array_equal(E.recall_per_query(ids, gt, 4), [0.5, 1.0])
    assert E.average_distance_ratio(np.array([[4.0, 9.0]]), np.array([[1.0, 9.0]]), 2) == 1.5  # (2 + 1) / 2
    assert E.average_distance_ratio(np.array([[1.0, 16.0]]), np.array([[0.0, 4.0]]), 2) == 2.0
    assert E.average_distance_ratio(np.array([[np.inf, 9.0]]), np.array([[1.0, 4.0]]), 2) == 1.5


def test_stop_model_and_training_state_files(tmp_path):
    """The stop network's file and Adam's state file round-trip exactly."""
    torch = pytest.importorskip("torch")
    from paper_2411_12229_gb300 import learned_stop as L
    P = torch.from_numpy(L.init_params(5))
    m = L.StopModel(P, 1.25, 8, 40, {"recall": 0.953, "train_queries": 20000})
    L.save_model(tmp_path / "stop.npz", m)
    r = L.load_model(tmp_path / "stop.npz", device="cpu")
    assert torch.equal(r.params, P) and (r.logit, r.every, r.ef_cap) == (1.25, 8, 40) and r.info == m.info
    np.savez(tmp_path / "bad.npz", params=np.zeros(7, np.float32), logit=0.0, every=1, ef_cap=1, info="{}")
    with pytest.raises(ValueError):
        L.load_model(tmp_path / "bad.npz", device="cpu")
    mm, vv = P * 0.5, P * P
    L.save_train_state(tmp_path / "st.npz", P, mm, vv, 77, 3)
    st = L.load_train_state(tmp_path / "st.npz")
    assert st["step"] == 77 and st["seed"] == 3
    np.testing.assert_array_equal(st["params"], P.numpy())
    np.testing.assert_array_equal(st["m"], mm.numpy())
    np.testing.assert_array_equal(st["v"], vv.numpy())


def test_build_graph_ex_on_the_host_equals_the_plain_call(lib_built):
    """sqg_build_graph_ex with device < 0 and no flags is sqg_build_graph;
    an unknown flag is an argument error; the host path reports every
    vertex as refined on the host."""
    from paper_2411_12229_gb300 import _binding as B
    rng = np.random.default_rng(12)
    n, d, R, L = 300, 64, 32, 48
    x = rng.standard_normal((n, d)).astype(np.float32)
    cand = rng.integers(0, n, (n, L)).astype(np.uint32)
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    a1, a2 = np.empty((n, R), np.uint32), np.empty((n, R), np.uint32)
    s1, s2 = np.zeros(5, np.uint64), np.zeros(5, np.uint64)
    assert B.lib().sqg_build_graph(ptr(x), n, d, ptr(cand), L, R, 0, 3, ptr(a1), ptr(s1), 2) == 0
    assert B.lib().sqg_build_graph_ex(ptr(x), n, d, ptr(cand), L, R, 0, 3, 0, ptr(a2), ptr(s2), 2, -1) == 0
    np.testing.assert_array_equal(a1, a2)
    np.testing.assert_array_equal(s1[:4], s2[:4])
    assert s2[4] == n
    assert B.lib().sqg_build_graph_ex(ptr(x), n, d, ptr(cand), L, R, 0, 3, 2, ptr(a2), ptr(s2), 2, -1) == -1


def test_serving_splits_ragged_batches_per_request():
    """The serving loop's result assembly: each retired batch's flat output
    (request sel[i]'s k results at the prefix sum of k over sel[:i]) goes
    back to its requests in any order of batches and requests."""
    from paper_2411_12229_gb300.serve import split_batches
    rng = np.random.default_rng(3)
    n = 40
    ks = rng.choice([1, 10, 100], size=n).astype(np.int32)
    want_i = [rng.integers(0, 1000, size=int(k)).astype(np.int32) for k in ks]
    want_d = [rng.random(int(k)).astype(np.float32) for k in ks]
    perm = rng.permutation(n)
    retired = []
    for part in np.array_split(perm, 5)[::-1]:  # batches retired out of order
        retired.append((part, np.concatenate([want_i[r] for r in part]), np.concatenate([want_d[r] for r in part])))
    got_i, got_d = split_batches(retired, ks, n + 1)
    for r in range(n):
        np.testing.assert_array_equal(got_i[r], want_i[r])
        np.testing.assert_array_equal(got_d[r], want_d[r])
    assert got_i[n] is None and got_d[n] is None

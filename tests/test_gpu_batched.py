"""The persistent batched form: autotuned launch knobs change nothing in the
results, and a CUDA-graph-captured batch replays the same search."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_every_tuning_knob_gives_identical_results(tiny_index, tmp_path, monkeypatch):
    from paper_2411_12229_gb300 import autotune
    from paper_2411_12229_gb300.api import Index
    monkeypatch.setenv("SQG_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    p, x, q = tiny_index
    ix = Index(p, 0)
    qd = torch.from_numpy(q).cuda()
    ref = ix.search(qd, 10, 64)
    cfgs = list(autotune.combos(ix))
    assert len(cfgs) == 36 + 2 * 12  # teams of 16 and 8 lanes only with the 96-register build
    for cfg in cfgs:
        got = ix.search(qd, 10, 64, **cfg)
        assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1]), cfg
    res = autotune.autotune(ix, qd, 10, 64, reps=2)
    assert len(res["table"]) == len(cfgs)
    assert autotune.tuned(ix, 64) == res["best"]
    assert autotune.tuned(ix, 1000) == autotune.DEFAULT


def test_graph_captured_batch_replays_the_search(tiny_index, oracle_mod):
    from paper_2411_12229_gb300.api import Index
    from paper_2411_12229_gb300.autotune import GraphSearch
    p, x, q = tiny_index
    ix = Index(p, 0)
    nq = 32
    rng = np.random.default_rng(2)
    k = rng.choice([1, 10, 30], size=nq).astype(np.int32)
    ef = (k * rng.integers(1, 5, size=nq)).astype(np.int32) + 8
    g = GraphSearch(ix, nq, k, ef, max_k=30, max_ef=int(ef.max()))
    off = np.concatenate([[0], np.cumsum(k)])
    O = oracle_mod.Index(p)
    for a in (0, 32):  # two replays with different queries
        ids, dists = g(torch.from_numpy(q[a:a + nq]).cuda())
        torch.cuda.synchronize()
        ids = ids.cpu().numpy().view(np.uint32)
        for i in range(nq):
            np.testing.assert_array_equal(ids[off[i]:off[i + 1]], O.search(q[a + i], int(k[i]), int(ef[i]))[0])


def test_host_pipeline_returns_each_batch_in_order(tiny_index, oracle_mod):
    """The pipelined host-to-host API: batches come back in submission
    order, each equal to the direct search of its queries."""
    from paper_2411_12229_gb300.api import Index
    p, x, q = tiny_index
    ix = Index(p, 0)
    nq = 16
    batches = [torch.from_numpy(np.ascontiguousarray(q[i * nq:(i + 1) * nq])).pin_memory() for i in range(4)]
    pipe = ix.host_pipeline(nq, 10, 48, depth=2)
    got = [r for r in (pipe.submit(b) for b in batches) if r is not None]
    got += pipe.drain()
    assert len(got) == len(batches)
    for b, (ids, dists) in zip(batches, got):
        ref_ids, ref_d = ix.search(b.cuda(), 10, 48)
        np.testing.assert_array_equal(ids, ref_ids.cpu().numpy())
        np.testing.assert_array_equal(dists, ref_d.cpu().numpy())
    assert pipe.drain() == []


def test_misaligned_pointers_are_rejected_before_any_launch(tiny_index):
    """Query rows are read as float4 and the workspace regions as uint4: a
    query pointer off a 16-byte boundary, or a workspace off 256 bytes, is
    an argument error caught on the host (nothing is launched)."""
    from paper_2411_12229_gb300 import _binding as B
    from paper_2411_12229_gb300.api import Index
    p, x, q = tiny_index
    ix = Index(p, 0)
    nq = 16
    qd = torch.from_numpy(q[:nq]).cuda()
    k = torch.full((nq,), 10, dtype=torch.int32, device="cuda")
    ef = torch.full((nq,), 32, dtype=torch.int32, device="cuda")
    ids = torch.empty(nq * 10, dtype=torch.int32, device="cuda")
    dd = torch.empty(nq * 10, dtype=torch.float32, device="cuda")
    ws = torch.empty(1 << 22, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    L = B.lib()
    # nq - 1 rows from one float in: in bounds even if it were read
    assert L.sqg_search_ex(ix.handle, qd.data_ptr() + 4, nq - 1, k.data_ptr(), ef.data_ptr(), ids.data_ptr(),
                           dd.data_ptr(), None, None, 0, None, s) == -1
    assert L.sqg_search_ex(ix.handle, qd.data_ptr(), nq, k.data_ptr(), ef.data_ptr(), ids.data_ptr(),
                           dd.data_ptr(), None, ws.data_ptr() + 16, ws.numel() - 16, None, s) == -1
    qr = torch.empty((nq, ix.d), dtype=torch.float32, device="cuda")
    pl = torch.empty((nq, 4, ix.d // 32), dtype=torch.int32, device="cuda")
    sc = torch.empty((nq, 4), dtype=torch.float32, device="cuda")
    assert L.sqg_prepare_queries(ix.handle, qd.data_ptr() + 4, nq - 1, qr.data_ptr(), pl.data_ptr(),
                                 sc.data_ptr(), s) == -1
    torch.cuda.synchronize()
    a = ix.search(qd, 10, 32)  # the aligned call still works
    assert a[0].shape == (nq, 10)

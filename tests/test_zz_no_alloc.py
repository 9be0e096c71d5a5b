"""sqg_search_noalloc: the search for callers that cannot allocate device
memory at search time (its scratch is a fixed array reserved when the
library loads).  Called through the C ABI and compared with sqg_search_ex
on two calls in a row -- the second call finds the first call's leftovers
in the shared array -- with the same bit-exact bar as the other parity
tests.  Collected last so that a failure here stops nothing else."""

import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _noalloc(ix, q, k, ef, max_k, max_ef):
    from paper_2411_12229_gb300 import _binding as B
    nq = q.shape[0]
    kt, et = k.cuda().int().contiguous(), ef.cuda().int().contiguous()
    total = int(k.sum())
    ids = torch.full((total,), -7, dtype=torch.int32, device="cuda")
    dists = torch.full((total,), -7.0, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = B.lib().sqg_search_noalloc(ix.handle, q.data_ptr(), nq, kt.data_ptr(), et.data_ptr(), max_k, max_ef,
                                    ids.data_ptr(), dists.data_ptr(), int(stream.cuda_stream))
    torch.cuda.synchronize()
    return rc, ids, dists


def test_noalloc_matches_search_ex_twice(tiny_index):
    from paper_2411_12229_gb300.api import Index
    p, x, qn = tiny_index
    ix = Index(p, 0)
    q = torch.from_numpy(qn).cuda()
    nq = q.shape[0]
    rng = np.random.default_rng(11)
    calls = [(np.full(nq, 10), np.full(nq, 64)),
             (rng.choice([1, 5, 20], size=nq), rng.integers(20, 97, size=nq))]
    for kk, ee in calls:  # two calls in a row on the same scratch
        k = torch.from_numpy(kk.astype(np.int32))
        ef = torch.from_numpy(np.maximum(ee, kk).astype(np.int32))
        rc, ids, dists = _noalloc(ix, q, k, ef, int(k.max()), int(ef.max()))
        assert rc == 0
        ref_ids, ref_d = ix.search(q, k, ef, max_k=int(k.max()), max_ef=int(ef.max()))
        torch.cuda.synchronize()
        assert torch.equal(ids, ref_ids)
        assert torch.equal(dists, ref_d)


def test_noalloc_rejects_a_batch_beyond_its_scratch(tiny_index):
    from paper_2411_12229_gb300 import _binding as B
    from paper_2411_12229_gb300.api import Index
    p, x, qn = tiny_index
    ix = Index(p, 0)
    limit = B.lib().sqg_noalloc_scratch_bytes()
    nq = 200_000  # 200k queries of d = 128 need more than the fixed scratch
    assert ix.workspace_size(nq, 10, 64) > limit
    q = torch.zeros((nq, ix.d), device="cuda")
    rc, _, _ = _noalloc(ix, q, torch.full((nq,), 10), torch.full((nq,), 64), 10, 64)
    assert rc == B.SqgError(-7).code == -7  # SQG_ERR_CAPACITY

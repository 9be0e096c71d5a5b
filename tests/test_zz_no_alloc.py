"""sqg_search_noalloc: the search for callers that cannot allocate device
memory at search time -- an application that reserved all GPU memory for
its own pool, a thread that must not enter the allocator mid-request.  Its
scratch is a fixed device array set up by its first call on a device.
Called through the C ABI and compared with sqg_search_ex on two calls in a
row -- the second call finds the first call's leftovers in the shared
array -- with the same bit-exact bar as the other parity tests: at small
beams, at a beam large enough that every query's visited set moves to the
array's full-size tables, and on a d = 512 index whose queries are rotated
on the tensor cores (their exactly quantized planes live in the array
too).  The device's stream-ordered pool is watched to show that the calls
allocate nothing.  Collected last so that a failure here stops nothing
else."""

import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8  # cuda.h: CUmemPool_attribute


class PoolWatch:
    """High watermark of the device's default stream-ordered pool (the
    pool cudaMallocAsync draws from), through the driver API."""

    def __init__(self, device: int):
        self.cu = C.CDLL("libcuda.so.1")
        dev = C.c_int()
        assert self.cu.cuDeviceGet(C.byref(dev), device) == 0
        self.pool = C.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(C.byref(self.pool), dev) == 0

    def reset(self):
        zero = C.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, C.byref(zero)) == 0

    def high(self) -> int:
        v = C.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, C.byref(v)) == 0
        return int(v.value)


def _noalloc(ix, q, k, ef, max_k, max_ef):
    from paper_2411_12229_gb300 import _binding as B
    nq = q.shape[0]
    kt, et = k.cuda().int().contiguous(), ef.cuda().int().contiguous()
    total = int(k.sum())
    ids = torch.full((max(total, 1),), -7, dtype=torch.int32, device="cuda")
    dists = torch.full((max(total, 1),), -7.0, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    rc = B.lib().sqg_search_noalloc(ix.handle, q.data_ptr(), nq, kt.data_ptr(), et.data_ptr(), max_k, max_ef,
                                    ids.data_ptr(), dists.data_ptr(), int(stream.cuda_stream))
    torch.cuda.synchronize()
    return rc, ids[:total], dists[:total]


def _check_twice(ix, q, calls, watch):
    for kk, ee in calls:  # two calls in a row on the same scratch
        k = torch.from_numpy(kk.astype(np.int32))
        ef = torch.from_numpy(np.maximum(ee, kk).astype(np.int32))
        watch.reset()
        rc, ids, dists = _noalloc(ix, q, k, ef, int(k.max()), int(ef.max()))
        assert rc == 0
        assert watch.high() == 0, "sqg_search_noalloc drew from the stream-ordered pool"
        ref_ids, ref_d, st = ix.search(q, k, ef, max_k=int(k.max()), max_ef=int(ef.max()), stats=True)
        torch.cuda.synchronize()
        assert torch.equal(ids, ref_ids)
        assert torch.equal(dists, ref_d)
    return st


def test_noalloc_matches_search_ex_twice(tiny_index):
    from paper_2411_12229_gb300.api import Index
    p, x, qn = tiny_index
    ix = Index(p, 0)
    watch = PoolWatch(0)
    q = torch.from_numpy(qn).cuda()
    nq = q.shape[0]
    # the set-up call (nq = 0) before anything else, as a pool-owning caller would
    rc, _, _ = _noalloc(ix, q[:0], torch.zeros(0, dtype=torch.int32), torch.zeros(0, dtype=torch.int32), 10, 64)
    assert rc == 0
    # the watch sees a search that does allocate (no workspace given)
    watch.reset()
    ix.search(q, 10, 64, max_k=10, max_ef=64)
    torch.cuda.synchronize()
    assert watch.high() > 0
    rng = np.random.default_rng(11)
    calls = [(np.full(nq, 10), np.full(nq, 64)),
             (rng.choice([1, 5, 20], size=nq), rng.integers(20, 97, size=nq))]
    _check_twice(ix, q, calls, watch)


def test_noalloc_visited_tables_in_the_scratch(tmp_path, lib_built):
    """Beams whose searches outgrow the 2^9 shared-memory visited slots: each
    query's visited set moves to its full-size table in the scratch array
    (cleared before use), on a 20,000-vertex index where such searches run
    long enough."""
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300 import synth
    from paper_2411_12229_gb300.api import Index
    w = synth.small(synth.BATCHED_1M_D128, 20000, 48)
    p = tmp_path / "n20k.sqg"
    ib.build_index(p, synth.base(w), 32, device=0, init="random", iterations=2, ef_build=64)
    ix = Index(p, 0)
    watch = PoolWatch(0)
    q = torch.from_numpy(synth.queries(w)).cuda()
    nq = q.shape[0]
    calls = [(np.full(nq, 10), np.full(nq, 2048)), (np.full(nq, 10), np.full(nq, 1500))]
    st = _check_twice(ix, q, calls, watch)
    # at least half of 2^9 expansions: the move happened (for nearly every query)
    assert float((st[:, 0] >= 256).float().mean()) >= 0.9


def test_noalloc_tensor_core_rotation(tmp_path, lib_built):
    """A d = 512 index: queries are rotated on the tensor cores and their
    exact 4-bit planes are written to the scratch array."""
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300 import synth
    from paper_2411_12229_gb300.api import Index
    w = synth.small(synth.HIGHDIM_1M_D960.with_(d=512), 1500, 48)
    x, qn = synth.base(w), synth.queries(w)
    p = tmp_path / "d512.sqg"
    ib.build_index(p, x, 32)
    ix = Index(p, 0)
    watch = PoolWatch(0)
    q = torch.from_numpy(qn).cuda()
    nq = q.shape[0]
    rng = np.random.default_rng(12)
    calls = [(np.full(nq, 10), np.full(nq, 80)), (rng.choice([1, 10], size=nq), rng.integers(10, 60, size=nq))]
    _check_twice(ix, q, calls, watch)


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

"""Teams of 16 and 8 lanes (2 and 4 queries per warp): the same search,
bit for bit, as the oracle's Algorithm 1 -- ids, distances, hop counts,
status and the expansion order -- across ef, out-degree 32 and 64, the
visited set's move to global memory, the ablations and a ragged batch."""

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


def _check(ix, O, q, k, ef, **kw):
    qd = torch.from_numpy(q).cuda()
    ids, dists, st = ix.search(qd, k, ef, stats=True, **kw)
    ids, dists, st = _np(ids).view(np.uint32), _np(dists), _np(st)
    okw = {a: kw[a] for a in ("eps0", "multi_estimate", "hop_cap") if a in kw}
    for i in range(q.shape[0]):
        oi, od, oh, os_ = O.search(q[i], k, ef, **okw)
        np.testing.assert_array_equal(ids[i], oi, err_msg=f"query {i} ids")
        np.testing.assert_array_equal(dists[i], od, err_msg=f"query {i} dists")
        assert (st[i, 0], st[i, 1]) == (oh, os_), f"query {i}: hops/status {st[i]} vs {(oh, os_)}"


@pytest.mark.parametrize("team", [16, 8])
@pytest.mark.parametrize("ef", [10, 33, 64, 300])
def test_team_parity_r32(gpu_tiny, oracle_mod, team, ef):
    ix, p, x, q = gpu_tiny
    _check(ix, oracle_mod.Index(p), q, 10, ef, team=team)


@pytest.mark.parametrize("team", [16, 8])
@pytest.mark.parametrize("ef", [16, 100])
def test_team_parity_r64(gpu_tiny64, oracle_mod, team, ef):
    ix, p, x, q = gpu_tiny64
    _check(ix, oracle_mod.Index(p), q, 10, ef, team=team)


@pytest.mark.parametrize("team", [16, 8])
def test_team_variants(gpu_tiny, oracle_mod, team):
    """eps0 > 0, without multiple estimates, a hop cap, the visited set moved
    to global memory early, the speculative prefetch, 1 and 2 warps per block."""
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    _check(ix, O, q, 10, 64, team=team, eps0=1.0)
    _check(ix, O, q, 10, 64, team=team, multi_estimate=False)
    _check(ix, O, q, 10, 64, team=team, hop_cap=20)
    _check(ix, O, q, 10, 128, team=team, visited_smem_log2=5)
    _check(ix, O, q, 10, 64, team=team, prefetch=2, warps_per_block=1)
    _check(ix, O, q, 10, 64, team=team, warps_per_block=2)


@pytest.mark.parametrize("team", [16, 8])
def test_team_expansion_order(gpu_tiny, oracle_mod, team):
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    r = ix.search_trace(torch.from_numpy(q).cuda(), 10, 64, None, 0, path_cap=512, team=team)
    st, path = _np(r[2]), _np(r[-1]).view(np.uint32)
    for i in range(q.shape[0]):
        opath = O.search(q[i], 10, 64, path_cap=512)[-1]
        assert st[i, 0] == len(opath)
        np.testing.assert_array_equal(path[i, :len(opath)], opath, err_msg=f"query {i}")
        assert np.all(path[i, len(opath):] == 0xFFFFFFFF)


@pytest.mark.parametrize("team", [16, 8])
def test_team_ragged_batch(gpu_tiny, oracle_mod, team):
    """Per-query k and ef, an odd batch size (teams of one warp end on
    different queries), invalid entries padded."""
    ix, p, x, q = gpu_tiny
    O = oracle_mod.Index(p)
    nq = 37
    rng = np.random.default_rng(5)
    k = rng.choice([1, 5, 10, 40], size=nq).astype(np.int32)
    ef = (k + rng.integers(0, 60, size=nq)).astype(np.int32)
    k[3] = 0  # invalid: padded, status flag
    qd = torch.from_numpy(q[:nq]).cuda()
    ids, dists, st = ix.search(qd, torch.from_numpy(k).cuda(), torch.from_numpy(ef).cuda(), stats=True, team=team,
                               max_k=40, max_ef=int(ef.max()))
    ids, dists, st = _np(ids).view(np.uint32), _np(dists), _np(st)
    off = np.concatenate([[0], np.cumsum(np.maximum(k, 0))])
    for i in range(nq):
        if k[i] < 1:
            continue
        oi, od, oh, os_ = O.search(q[i], int(k[i]), int(ef[i]))
        np.testing.assert_array_equal(ids[off[i]:off[i + 1]], oi, err_msg=f"query {i}")
        np.testing.assert_array_equal(dists[off[i]:off[i + 1]], od)
        assert st[i, 0] == oh
    assert st[3, 1] == 4 and ix.status() & 4  # the invalid entry, flag read and cleared


def test_team_rejects_stop_network_and_large_d(gpu_tiny, shaped_index_file):
    from paper_2411_12229_gb300 import _binding as B
    from paper_2411_12229_gb300.api import Index
    ix, p, x, q = gpu_tiny
    qd = torch.from_numpy(q).cuda()
    mlp = torch.zeros(B.MLP_NPARAM, device="cuda")
    with pytest.raises(B.SqgError):
        ix.search(qd, 10, 64, team=16, stop_mlp=mlp)
    with pytest.raises(B.SqgError):
        ix.search(qd, 10, 64, team=12)
    p2, x2, q2 = shaped_index_file
    ix2 = Index(p2, 0)
    if ix2.d > 256:
        with pytest.raises(B.SqgError):
            ix2.search(torch.from_numpy(q2).cuda(), 10, 40, team=16)

"""Sharded search: an index split into S shards, each with its own graph.

Not in the paper, whose scalability study (Sec. 5, Deep-100M and
MSTuring-100M) keeps one graph per index.  When an index outgrows one GPU,
the vectors are split into S contiguous shards, Algorithm 2 builds a graph
on each shard alone, and a query is searched in every shard (Algorithm 1);
the per-shard top-k lists, sorted by (distance, id), are then merged into
one global top-k by ``sqg_merge_topk`` (a CUDA kernel).  Results can differ
from one graph over all vectors: each shard's beam explores its own graph.

Placement: rank r of W ranks holds shards [r S/W, (r+1) S/W) (S a multiple
of W).  One rank (W = 1) searches every shard on its GPU in turn; with
W > 1 each rank searches its own shards and one all-gather of the k x 8
bytes per query per shard (``exchange``) gives every rank all lists, which
it merges itself.  The search on the data path is the library's; only the
exchange is a collective.
"""

from __future__ import annotations

import ctypes as C
import json
import pathlib

import numpy as np

from . import _binding as B


def shard_ranges(n: int, shards: int) -> list[tuple[int, int]]:
    """Contiguous, balanced row ranges [lo, hi) of the S shards."""
    if shards < 1 or shards > min(n, B.MAX_SHARDS):
        raise ValueError(f"need 1 <= shards <= min(n, {B.MAX_SHARDS})")
    return [(s * n // shards, (s + 1) * n // shards) for s in range(shards)]


def build_shards(prefix, data: np.ndarray, R: int, shards: int, **build_kw) -> pathlib.Path:
    """One index file per shard (its own graph, Algorithm 2) plus a manifest
    (``<prefix>.shards.json``: files, row ranges, global id offsets)."""
    from . import index_builder as ib
    prefix = pathlib.Path(prefix)
    ranges = shard_ranges(data.shape[0], shards)
    files = []
    for s, (lo, hi) in enumerate(ranges):
        f = prefix.parent / f"{prefix.name}.shard{s}.sqg"
        ib.build_index(f, np.ascontiguousarray(data[lo:hi]), R, **build_kw)
        files.append(f.name)
    man = prefix.parent / f"{prefix.name}.shards.json"
    man.write_text(json.dumps({"shards": shards, "n": int(data.shape[0]), "files": files,
                               "ranges": ranges, "offsets": [lo for lo, _ in ranges]}, indent=1))
    return man


def load_manifest(path) -> dict:
    path = pathlib.Path(path)
    m = json.loads(path.read_text())
    m["paths"] = [path.parent / f for f in m["files"]]
    return m


def exchange(ids, dists, group=None):
    """All-gather of every rank's per-shard lists ([S_local, nq, k] ids and
    distances) into [S, nq, k] in shard order; NCCL for device tensors,
    gloo for host tensors."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    gi = [torch.empty_like(ids) for _ in range(world)]
    gd = [torch.empty_like(dists) for _ in range(world)]
    dist.all_gather(gi, ids.contiguous(), group=group)
    dist.all_gather(gd, dists.contiguous(), group=group)
    return torch.cat(gi, 0), torch.cat(gd, 0)


class ShardedIndex:
    """The shards this rank holds, loaded on one GPU, and the search over
    all shards with the merge."""

    def __init__(self, manifest, device: int = 0, rank: int = 0, world: int = 1, group=None):
        from .api import Index
        m = load_manifest(manifest)
        S = m["shards"]
        if S % world:
            raise ValueError("the shard count must be a multiple of the rank count")
        per = S // world
        self.S, self.rank, self.world, self.group, self.device = S, rank, world, group, device
        self.offsets = np.asarray(m["offsets"], dtype=np.uint32)
        self.local = list(range(rank * per, (rank + 1) * per))
        self.shards = [Index(m["paths"][s], device) for s in self.local]
        self.d = self.shards[0].d

    def close(self):
        for ix in self.shards:
            ix.close()

    def search(self, queries, k: int, ef: int, **kw):
        """Top-k of every query over all shards: (ids int32, dists float32),
        (nq, k), global ids sorted by (distance, id); padding -1 / +inf."""
        import torch
        nq = queries.shape[0]
        dev = queries.device
        li = torch.empty((len(self.shards), nq, k), dtype=torch.int32, device=dev)
        ld = torch.empty((len(self.shards), nq, k), dtype=torch.float32, device=dev)
        for j, ix in enumerate(self.shards):
            ix.search(queries, k, ef, out=(li[j].view(-1), ld[j].view(-1)), max_k=k, max_ef=ef, **kw)
        if self.world > 1:
            li, ld = exchange(li, ld, self.group)
        return merge_topk(li, ld, self.offsets, k)


def merge_topk(ids, dists, offsets, k: int, stream=None):
    """sqg_merge_topk over [S, nq, k] device lists with host offsets."""
    import torch
    S, nq = ids.shape[0], ids.shape[1]
    out_i = torch.empty((nq, k), dtype=torch.int32, device=ids.device)
    out_d = torch.empty((nq, k), dtype=torch.float32, device=ids.device)
    off = np.ascontiguousarray(offsets, dtype=np.uint32)
    s = stream if stream is not None else torch.cuda.current_stream(ids.device)
    B.check(B.lib().sqg_merge_topk(ids.contiguous().data_ptr(), dists.contiguous().data_ptr(), S, nq, k,
                                   off.ctypes.data_as(C.c_void_p), out_i.data_ptr(), out_d.data_ptr(),
                                   int(s.cuda_stream)), "sqg_merge_topk")
    return out_i, out_d

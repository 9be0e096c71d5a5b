"""Autotuner for the search kernel's launch knobs (not in the paper).

Knobs, all result-neutral (the search is bit-identical under each):
  warps_per_block    query-warps per block (occupancy granularity)
  prefetch           1: the next block copied into shared memory during
                     the merge; 2: also L2-prefetch the runner-up's block
  visited_smem_log2  shared-memory slots of the visited set (2^9, 2^10)
  lean               0 / 1: the search kernel's builds for fewer / more
                     resident warps (d <= 256; 1 caps the registers lower,
                     with a few spills); 2: the general kernel's
                     96-register build
  team               lanes per query: 32, or 16 / 8 with 2 / 4 queries per
                     warp (d <= 256; always the 96-register build)
The tuner times every combination on the caller's own batch (CUDA events,
median of `reps`) and keeps the fastest per (GPU, d, R, ef bucket) in a
JSON cache, which ``tuned`` then returns.

``GraphSearch`` captures one fixed-shape batched search (persistent kernel,
caller workspace, explicit bounds, so nothing allocates or synchronizes)
into a CUDA graph and replays it.
"""

from __future__ import annotations

import itertools
import json
import os
import pathlib

import numpy as np
import torch

KNOBS = {"warps_per_block": (1, 2, 4), "prefetch": (1, 2), "visited_smem_log2": (9, 10), "lean": (0, 1, 2),
         "team": (32, 16, 8)}
DEFAULT = {"warps_per_block": 4, "prefetch": 1, "visited_smem_log2": 0, "lean": 0, "team": 0}


def combos(ix, knobs=None):
    """The knob combinations that apply to this index (teams below 32 lanes
    only for d <= 256, where the register build is fixed)."""
    knobs = knobs or KNOBS
    names = list(knobs)
    for combo in itertools.product(*(knobs[n] for n in names)):
        cfg = dict(zip(names, combo))
        if cfg.get("team", 32) < 32 and (ix.d > 256 or cfg.get("lean", 2) != 2):
            continue
        yield cfg


def cache_path() -> pathlib.Path:
    return pathlib.Path(os.environ.get("SQG_AUTOTUNE_CACHE", pathlib.Path.home() / ".cache" / "sqg_autotune.json"))


def _key(ix, ef: int) -> str:
    bucket = 1 << int(np.ceil(np.log2(max(1, ef))))
    return f"{torch.cuda.get_device_name(ix.device)}|d{ix.d}|R{ix.degree}|ef{bucket}"


def _time(ix, q, k, ef, reps, **kw) -> float:
    ix.search(q, k, ef, **kw)
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ix.search(q, k, ef, **kw)
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return float(np.median(ms))


def autotune(ix, queries: torch.Tensor, k, ef, *, reps: int = 5, save: bool = True, knobs=None) -> dict:
    """Time every knob combination; returns {"best": {...}, "table": [...]}."""
    knobs = knobs or KNOBS
    names = list(knobs)
    table = []
    efmax = int(ef) if np.ndim(ef) == 0 else int(torch.as_tensor(ef).max())
    for cfg in combos(ix, knobs):
        ms = _time(ix, queries, k, ef, reps, **cfg)
        table.append({**cfg, "ms": round(ms, 4), "qps": round(queries.shape[0] / (ms / 1e3))})
    best = min(table, key=lambda r: r["ms"])
    out = {"best": {n: best[n] for n in names}, "table": table}
    if save:
        p = cache_path()
        p.parent.mkdir(parents=True, exist_ok=True)
        db = json.loads(p.read_text()) if p.exists() else {}
        db[_key(ix, efmax)] = out["best"]
        p.write_text(json.dumps(db, indent=1))
    return out


def tuned(ix, ef: int) -> dict:
    """The cached best knobs for this index and ef (defaults if untuned)."""
    p = cache_path()
    if p.exists():
        db = json.loads(p.read_text())
        v = db.get(_key(ix, ef))
        if v:
            return dict(v)
    return dict(DEFAULT)


class GraphSearch:
    """One batched search of fixed shape captured as a CUDA graph."""

    def __init__(self, ix, nq: int, k, ef, *, max_k: int, max_ef: int, **kw):
        self.ix = ix
        dev = torch.device("cuda", ix.device)
        self.q = torch.zeros((nq, ix.d), dtype=torch.float32, device=dev)
        self.k = torch.as_tensor(np.broadcast_to(np.asarray(k, dtype=np.int32), (nq,)).copy(), device=dev)
        self.ef = torch.as_tensor(np.broadcast_to(np.asarray(ef, dtype=np.int32), (nq,)).copy(), device=dev)
        total = int(self.k.sum())
        self.ids = torch.empty(total, dtype=torch.int32, device=dev)
        self.dists = torch.empty(total, dtype=torch.float32, device=dev)
        self.ws = torch.empty(ix.workspace_size(nq, max_k, max_ef, **kw), dtype=torch.uint8, device=dev)
        self.kw = dict(max_k=max_k, max_ef=max_ef, **kw)
        if np.ndim(k) == 0 and "uniform_k" not in kw and max_k == int(k):
            self.kw["uniform_k"] = int(k)  # one k: outputs at i * k, no planning kernel
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):  # warm-up outside the capture
            self._run(s)
        torch.cuda.current_stream(dev).wait_stream(s)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._run(torch.cuda.current_stream(dev))

    def _run(self, stream):
        self.ix.search(self.q, self.k, self.ef, out=(self.ids, self.dists), workspace=self.ws, stream=stream,
                       **self.kw)

    def __call__(self, queries: torch.Tensor | None = None):
        if queries is not None:
            self.q.copy_(queries)
        self.graph.replay()
        return self.ids, self.dists

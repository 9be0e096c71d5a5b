"""Continuous-batching request loop over the search kernel (not in the paper).

Requests (a query, its k and ef) arrive over time.  The loop admits every
request that has arrived while (a) a stream slot is free and (b) the device
memory its search needs fits the budget; admitted requests go out as one
batched launch on one of several CUDA streams, so batches launched while
others still run overlap on the device.  A batch releases its memory and
its slot when its completion event fires; each request's latency is its
completion time minus its arrival time.

Memory per request (the admission unit) is what the search holds for it:
beam ef x 8 B, result k x 8 B, visited hash 4 x 2^ceil(log2(2(4 ef + 64)+1))
B, the rotated query 4d B and its offset/stats (16 B), plus its output.
The search is deterministic per query, so a request's result is the same
alone and in any mix (tested).
"""

from __future__ import annotations

import dataclasses
import math
import time

import numpy as np
import torch


def request_bytes(k: int, ef: int, d: int) -> int:
    cap = 4 * ef + 64
    hb = 4 << max(5, math.ceil(math.log2(2 * cap + 1)))
    return 8 * ef + 8 * k + hb + 4 * d + 16 + 8 * k


@dataclasses.dataclass
class ServeResult:
    latency_s: np.ndarray   # per request
    done_at_s: np.ndarray   # completion time (from the start of the run)
    ids: list               # per request: np.ndarray of k ids
    dists: list
    batches: int
    max_inflight_bytes: int
    wall_s: float

    def summary(self) -> dict:
        lat = self.latency_s * 1e3
        span = float(self.done_at_s.max() - self.done_at_s.min()) if len(lat) > 1 else self.wall_s
        return {"requests": int(len(lat)), "qps": round(len(lat) / max(self.wall_s, 1e-9), 1),
                "p50_ms": round(float(np.percentile(lat, 50)), 4), "p99_ms": round(float(np.percentile(lat, 99)), 4),
                "mean_ms": round(float(lat.mean()), 4), "batches": self.batches,
                "max_inflight_bytes": self.max_inflight_bytes, "span_s": round(span, 4)}


class Server:
    """Continuous batching over `streams` CUDA streams on one index."""

    def __init__(self, ix, *, max_k: int, max_ef: int, mem_budget: int = 256 << 20, streams: int = 4,
                 max_batch: int = 8192, stop_model=None):
        self.ix = ix
        self.max_k, self.max_ef = max_k, max_ef
        self.mem_budget = mem_budget
        self.max_batch = max_batch
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.stop = stop_model
        d = ix.d
        ws = ix.workspace_size(max_batch, max_k, max_ef)
        self.slots = []
        for s in self.streams:
            self.slots.append(dict(
                stream=s,
                ws=torch.empty(ws, dtype=torch.uint8, device="cuda"),
                qh=torch.empty((max_batch, d), dtype=torch.float32).pin_memory(),
                kh=torch.empty(max_batch, dtype=torch.int32).pin_memory(),
                eh=torch.empty(max_batch, dtype=torch.int32).pin_memory(),
                ih=torch.empty(max_batch * max_k, dtype=torch.int32).pin_memory(),
                dh=torch.empty(max_batch * max_k, dtype=torch.float32).pin_memory(),
                ids=torch.empty(max_batch * max_k, dtype=torch.int32, device="cuda"),
                dists=torch.empty(max_batch * max_k, dtype=torch.float32, device="cuda"),
                busy=None))

    def _launch(self, slot, sel, queries, ks, efs):
        n = len(sel)
        slot["qh"][:n].copy_(torch.from_numpy(queries[sel]))
        slot["kh"][:n].copy_(torch.from_numpy(ks[sel]))
        slot["eh"][:n].copy_(torch.from_numpy(efs[sel]))
        s = slot["stream"]
        with torch.cuda.stream(s):
            qd = slot["qh"][:n].to("cuda", non_blocking=True)
            kd = slot["kh"][:n].to("cuda", non_blocking=True)
            ed = slot["eh"][:n].to("cuda", non_blocking=True)
            kw = {}
            if self.stop is not None:
                kw = dict(stop_mlp=self.stop.params, stop_logit=self.stop.logit, stop_every=self.stop.every)
            tot = int(ks[sel].sum())
            self.ix.search(qd, kd, ed, out=(slot["ids"][:tot], slot["dists"][:tot]), workspace=slot["ws"],
                           max_k=self.max_k, max_ef=self.max_ef, stream=s, **kw)
            slot["ih"][:tot].copy_(slot["ids"][:tot], non_blocking=True)
            slot["dh"][:tot].copy_(slot["dists"][:tot], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        # keep the device tensors alive until the batch completes
        slot["busy"] = (ev, sel, tot, (qd, kd, ed))

    def run(self, queries: np.ndarray, ks: np.ndarray, efs: np.ndarray, arrivals_s: np.ndarray) -> ServeResult:
        n = queries.shape[0]
        order = np.argsort(arrivals_s, kind="stable")
        need = np.array([request_bytes(int(k), int(e), self.ix.d) for k, e in zip(ks, efs)], dtype=np.int64)
        lat = np.zeros(n)
        done_at = np.zeros(n)
        out_ids, out_d = [None] * n, [None] * n
        nxt = 0            # next request (in arrival order) not yet admitted
        inflight = 0       # bytes held by running batches
        held = {}          # slot index -> bytes
        peak, batches, finished = 0, 0, 0
        queries = np.ascontiguousarray(queries, dtype=np.float32)
        ks = np.ascontiguousarray(ks, dtype=np.int32)
        efs = np.ascontiguousarray(efs, dtype=np.int32)
        t0 = time.perf_counter()
        while finished < n:
            now = time.perf_counter() - t0
            progressed = False
            for si, slot in enumerate(self.slots):  # retire completed batches
                b = slot["busy"]
                if b is not None and b[0].query():
                    tdone = time.perf_counter() - t0
                    ev, sel, tot, _ = b
                    ih, dh = slot["ih"][:tot].numpy(), slot["dh"][:tot].numpy()
                    off = 0
                    for r in sel:
                        kk = int(ks[r])
                        out_ids[r], out_d[r] = ih[off:off + kk].copy(), dh[off:off + kk].copy()
                        off += kk
                        lat[r] = tdone - arrivals_s[r]
                        done_at[r] = tdone
                    finished += len(sel)
                    inflight -= held.pop(si)
                    slot["busy"] = None
                    progressed = True
            for si, slot in enumerate(self.slots):  # admit arrived requests
                if slot["busy"] is not None or nxt >= n or arrivals_s[order[nxt]] > now:
                    continue
                sel, budget = [], self.mem_budget - inflight
                while (nxt < n and len(sel) < self.max_batch and arrivals_s[order[nxt]] <= now
                       and need[order[nxt]] <= budget):
                    r = order[nxt]
                    sel.append(r)
                    budget -= need[r]
                    nxt += 1
                if not sel:
                    break  # memory full: wait for a completion
                b = int(need[sel].sum())
                held[si] = b
                inflight += b
                peak = max(peak, inflight)
                self._launch(slot, np.array(sel), queries, ks, efs)
                batches += 1
                progressed = True
            if not progressed:
                if nxt < n and all(s["busy"] is None for s in self.slots):
                    wait = arrivals_s[order[nxt]] - (time.perf_counter() - t0)
                    if wait > 2e-4:
                        time.sleep(wait - 1e-4)
                else:
                    time.sleep(2e-5)
        wall = time.perf_counter() - t0
        return ServeResult(lat, done_at, out_ids, out_d, batches, peak, wall)


def main():
    """Offered-load sweep on the serving workload: p50/p99 latency and QPS."""
    import argparse
    import json
    import os
    import pathlib
    import sys

    sys.path.insert(0, str(pathlib.Path(__file__).resolve().parents[1]))
    from . import eval as E
    from . import index_builder as ib
    from . import synth
    from .api import Index

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="serving-4m-d96")
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--loads", default="50000,100000,200000,500000,1000000,2000000")
    ap.add_argument("--seconds", type=float, default=1.0)
    ap.add_argument("--cache", default=os.environ.get("SQG_CACHE", "/tmp/sqg_cache"))
    ap.add_argument("--mem-mb", type=int, default=256)
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--target", type=float, default=0.95)
    args = ap.parse_args()
    w = synth.WORKLOADS[args.workload]
    if args.n:
        w = synth.small(w, args.n, w.n_queries)
    cache = pathlib.Path(args.cache)
    cache.mkdir(parents=True, exist_ok=True)
    path = cache / f"{w.name}-n{w.n}-R{w.degree}-it3-ef400.sqg"
    if not path.exists():
        base = synth.base(w)
        ib.build_index(str(path) + ".part", base, w.degree, device=0, init="random", iterations=3, ef_build=400)
        os.replace(str(path) + ".part", path)
    else:
        base = None
    ix = Index(path, 0)
    q = synth.queries(w)
    base = synth.base(w) if base is None else base
    gt, _ = E.ground_truth(base, q, 100, device=0)
    qd = torch.from_numpy(q).cuda()
    # ef per k calibrated on the test queries: the smallest ef reaching the
    # target recall@k (k = 10 and k = 100)
    ef_for = {}
    for k in (10, 100):
        for ef in [e for e in synth.EF_SWEEP if e >= k] + [768, 1024]:
            ids, _ = ix.search(qd, k, ef)
            if E.recall(ids.cpu().numpy(), gt, k) >= args.target:
                break
        ef_for[k] = ef
    res = {"workload": w.name, "n": w.n, "ef_for_k": ef_for, "loads": []}
    srv = Server(ix, max_k=100, max_ef=max(ef_for.values()), mem_budget=args.mem_mb << 20,
                 streams=args.streams, max_batch=8192)
    rng = np.random.default_rng(5)
    for load in [int(x) for x in args.loads.split(",")]:
        m = int(min(200_000, max(2000, load * args.seconds)))
        sel = rng.integers(0, q.shape[0], size=m)
        ks = np.where(rng.integers(0, 2, size=m) == 0, 10, 100).astype(np.int32)
        efs = np.array([ef_for[int(k)] for k in ks], dtype=np.int32)
        arr = synth.poisson_arrivals(float(load), m)
        r = srv.run(q[sel], ks, efs, arr)
        s = r.summary()
        hit = [len(np.intersect1d(r.ids[i], gt[sel[i], :10])) / 10 for i in range(m) if ks[i] == 10]
        s.update(offered_qps=load, recall_at_10=round(float(np.mean(hit)), 4))
        res["loads"].append(s)
        print(json.dumps(s), flush=True)
    print(json.dumps(res))


if __name__ == "__main__":
    main()

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
alone and in any mix (tested).  The offered-load sweep on the serving
workload is `python bench.py --workload serving-4m-d96`.
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


def split_batches(retired, ks: np.ndarray, n: int):
    """Per-request (ids, dists) from retired batches.  Each batch is
    (sel, flat_ids, flat_dists): the requests it served, in launch order,
    and its ragged output, request sel[i]'s k results starting at the sum
    of the k of sel[:i] (the search's output layout).  Returns two lists of
    n arrays (views into the batches' arrays), None for a request no batch
    served."""
    out_ids, out_d = [None] * n, [None] * n
    for sel, bi, bd in retired:
        kk = ks[sel]
        ends = np.cumsum(kk)
        for r, a, e in zip(sel, ends - kk, ends):
            out_ids[r], out_d[r] = bi[a:e], bd[a:e]
    return out_ids, out_d


@dataclasses.dataclass
class ServeResult:
    latency_s: np.ndarray   # per request
    done_at_s: np.ndarray   # completion time (from the start of the run)
    ids: list               # per request: np.ndarray of k ids
    dists: list
    batches: int
    max_inflight_bytes: int
    wall_s: float
    search_ms: float = 0.0  # device time of the batches' searches (events around each launch), summed
    loop_s: float = 0.0     # host time spent admitting, launching and retiring (the loop's own work)

    def summary(self) -> dict:
        lat = self.latency_s * 1e3
        span = float(self.done_at_s.max() - self.done_at_s.min()) if len(lat) > 1 else self.wall_s
        return {"requests": int(len(lat)), "qps": round(len(lat) / max(self.wall_s, 1e-9), 1),
                "p50_ms": round(float(np.percentile(lat, 50)), 4), "p99_ms": round(float(np.percentile(lat, 99)), 4),
                "mean_ms": round(float(lat.mean()), 4), "batches": self.batches,
                "mean_batch": round(len(lat) / max(self.batches, 1), 1),
                "max_inflight_bytes": self.max_inflight_bytes, "span_s": round(span, 4),
                "device_search_s": round(self.search_ms / 1e3, 4), "host_loop_s": round(self.loop_s, 4)}


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
        # gathered straight into the pinned staging buffers (no temporaries)
        np.take(queries, sel, axis=0, out=slot["qh"][:n].numpy())
        np.take(ks, sel, out=slot["kh"][:n].numpy())
        np.take(efs, sel, out=slot["eh"][:n].numpy())
        s = slot["stream"]
        with torch.cuda.stream(s):
            qd = slot["qh"][:n].to("cuda", non_blocking=True)
            kd = slot["kh"][:n].to("cuda", non_blocking=True)
            ed = slot["eh"][:n].to("cuda", non_blocking=True)
            kw = {}
            if self.stop is not None:
                kw = dict(stop_mlp=self.stop.params, stop_logit=self.stop.logit, stop_every=self.stop.every)
            tot = int(slot["kh"][:n].numpy().sum())
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            self.ix.search(qd, kd, ed, out=(slot["ids"][:tot], slot["dists"][:tot]), workspace=slot["ws"],
                           max_k=self.max_k, max_ef=self.max_ef, stream=s, **kw)
            e1.record(s)
            slot["ih"][:tot].copy_(slot["ids"][:tot], non_blocking=True)
            slot["dh"][:tot].copy_(slot["dists"][:tot], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        # keep the device tensors alive until the batch completes
        slot["busy"] = (ev, sel, tot, (qd, kd, ed), (e0, e1))

    def run(self, queries: np.ndarray, ks: np.ndarray, efs: np.ndarray, arrivals_s: np.ndarray) -> ServeResult:
        """Serve requests (query, k, ef) arriving at arrivals_s seconds from
        the start.  Admission and retirement are vectorized over the
        requests they move, so the host loop's cost per request stays small
        next to the search's."""
        n = queries.shape[0]
        order = np.argsort(arrivals_s, kind="stable")
        arr_sorted = np.asarray(arrivals_s, dtype=np.float64)[order]
        need = np.array([request_bytes(int(k), int(e), self.ix.d) for k, e in zip(ks, efs)], dtype=np.int64)
        cum_need = np.concatenate([[0], np.cumsum(need[order])])  # bytes of the first i requests in arrival order
        lat = np.zeros(n)
        done_at = np.zeros(n)
        ks = np.ascontiguousarray(ks, dtype=np.int32)
        efs = np.ascontiguousarray(efs, dtype=np.int32)
        retired = []       # per batch: (requests, their flat ids, dists), split per request after the loop
        nxt = 0            # next request (in arrival order) not yet admitted
        inflight = 0       # bytes held by running batches
        held = {}          # slot index -> bytes
        peak, batches, finished = 0, 0, 0
        search_ms, idle_s = 0.0, 0.0
        queries = np.ascontiguousarray(queries, dtype=np.float32)
        t0 = time.perf_counter()
        while finished < n:
            now = time.perf_counter() - t0
            progressed = False
            for si, slot in enumerate(self.slots):  # retire completed batches
                b = slot["busy"]
                if b is not None and b[0].query():
                    tdone = time.perf_counter() - t0
                    ev, sel, tot, _, (e0, e1) = b
                    search_ms += e0.elapsed_time(e1)
                    retired.append((sel, slot["ih"][:tot].numpy().copy(), slot["dh"][:tot].numpy().copy()))
                    lat[sel] = tdone - arrivals_s[sel]
                    done_at[sel] = tdone
                    finished += len(sel)
                    inflight -= held.pop(si)
                    slot["busy"] = None
                    progressed = True
            for si, slot in enumerate(self.slots):  # admit arrived requests
                if slot["busy"] is not None or nxt >= n or arr_sorted[nxt] > now:
                    continue
                arrived = int(np.searchsorted(arr_sorted, now, side="right"))
                fit = int(np.searchsorted(cum_need, cum_need[nxt] + self.mem_budget - inflight, side="right")) - 1
                end = min(arrived, fit, nxt + self.max_batch)
                if end <= nxt:
                    break  # memory full: wait for a completion
                sel = order[nxt:end]
                b = int(cum_need[end] - cum_need[nxt])
                nxt = end
                held[si] = b
                inflight += b
                peak = max(peak, inflight)
                self._launch(slot, sel, queries, ks, efs)
                batches += 1
                progressed = True
            if not progressed:
                ts = time.perf_counter()
                if nxt < n and all(s["busy"] is None for s in self.slots):
                    wait = arr_sorted[nxt] - (time.perf_counter() - t0)
                    if wait > 2e-4:
                        time.sleep(wait - 1e-4)
                else:
                    time.sleep(2e-5)
                idle_s += time.perf_counter() - ts
        wall = time.perf_counter() - t0
        out_ids, out_d = split_batches(retired, ks, n)
        return ServeResult(lat, done_at, out_ids, out_d, batches, peak, wall, search_ms, wall - idle_s)

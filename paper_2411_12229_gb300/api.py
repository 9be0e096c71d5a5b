"""Python face of libsqg: a thin wrapper over the C ABI (include/sqg.h).

Device memory and streams come from PyTorch; every step of the search runs
in the library's kernels.  Tensors are passed by ``data_ptr()`` and the
current CUDA stream is used unless one is given.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import _binding as B


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _i32(x, nq: int, device) -> torch.Tensor:
    if isinstance(x, torch.Tensor):
        t = x.to(device=device, dtype=torch.int32).contiguous()
    else:
        t = torch.as_tensor(np.broadcast_to(np.asarray(x, dtype=np.int32), (nq,)).copy(), device=device)
    if t.numel() != nq:
        raise ValueError(f"expected {nq} values, got {t.numel()}")
    return t


class Index:
    """A SymphonyQG index resident on one GPU (sqg_index_load)."""

    def __init__(self, path: str | os.PathLike, device: int | None = None):
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = C.c_void_p()
        B.check(B.lib().sqg_index_load(str(path).encode(), self.device, C.byref(h)), f"sqg_index_load({path})")
        self._h = h
        info = B.Info()
        B.check(B.lib().sqg_index_info(h, C.byref(info)), "sqg_index_info")
        self.n, self.d, self.degree = int(info.n), int(info.d), int(info.degree)
        self.block_bytes, self.entry = int(info.block_bytes), int(info.entry)
        self.device_bytes = int(info.device_bytes)
        self.fjlt = int(info.version) == 2  # the fast JLT (data zero-padded to d)
        # "l2" (squared Euclidean) or "cosine" (unit vectors; queries are
        # normalized by the library, distances are 2 - 2 cos)
        self.metric = "cosine" if int(info.metric) == 1 else "l2"

    def fit_queries(self, queries: torch.Tensor) -> torch.Tensor:
        """Queries of a fast-JLT index may have fewer columns than d (the data
        were zero-padded to a power of 2): pad them the same way."""
        if queries.dim() == 2 and queries.shape[1] < self.d and self.fjlt:
            return torch.nn.functional.pad(queries, (0, self.d - queries.shape[1]))
        return queries

    def close(self) -> None:
        if getattr(self, "_h", None):
            B.lib().sqg_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> C.c_void_p:
        return self._h

    # ------------------------------------------------------------------ search
    def params(self, *, eps0: float = 0.0, multi_estimate: bool = True, hop_cap: int = 0, max_k: int = 0,
               max_ef: int = 0, stop_mlp: torch.Tensor | None = None, stop_logit: float = 0.0,
               stop_every: int = 1, warps_per_block: int = 0, timing_events=None, visited_smem_log2: int = 0,
               prefetch: int = 0, lean: int = 0, rotation: int = 0, team: int = 0,
               kernel: int = 0, uniform_k: int = 0) -> B.SearchParams:
        p = B.SearchParams()
        p.eps0 = float(eps0)
        p.multi_estimate = 1 if multi_estimate else 0
        p.hop_cap = int(hop_cap)
        p.max_k, p.max_ef = int(max_k), int(max_ef)
        if stop_mlp is not None:
            if stop_mlp.dtype != torch.float32 or not stop_mlp.is_cuda or stop_mlp.numel() != B.MLP_NPARAM:
                raise ValueError("stop_mlp must be a CUDA float32 tensor of 5313 parameters")
            p.stop_mlp = stop_mlp.data_ptr()
        p.stop_logit = float(stop_logit)
        p.stop_every = int(stop_every)
        p.warps_per_block = int(warps_per_block)
        p.visited_smem_log2 = int(visited_smem_log2)
        p.prefetch = int(prefetch)
        p.lean = int(lean)
        p.rotation = int(rotation)
        p.team = int(team)
        p.kernel = int(kernel)
        p.uniform_k = int(uniform_k)
        if timing_events is not None:  # torch.cuda.Event pair, already recorded once
            p.timing_events[0] = timing_events[0].cuda_event
            p.timing_events[1] = timing_events[1].cuda_event
        return p

    def search(self, queries: torch.Tensor, k, ef, *, out: tuple | None = None, stats: bool = False,
               workspace: torch.Tensor | None = None, stream=None, **kw):
        """Search a batch (Algorithm 1 per query).

        queries: (nq, d) float32 CUDA tensor.  k, ef: ints or (nq,) tensors.
        Returns (ids int32, dists float32): shape (nq, k) when k is one int
        (or (nq, uniform_k) with that keyword), else flat ragged arrays
        (query i at offset sum_{j<i} k[j]).  Padding
        is id -1 with distance +inf.  With stats=True also returns an
        (nq, 2) int32 tensor of (hops, status bits)."""
        queries = self.fit_queries(queries)
        if queries.dtype != torch.float32 or not queries.is_cuda or queries.dim() != 2 or queries.shape[1] != self.d:
            raise ValueError(f"queries must be a CUDA float32 tensor of shape (nq, {self.d})")
        queries = queries.contiguous()
        nq, dev = queries.shape[0], queries.device
        kt, et = _i32(k, nq, dev), _i32(ef, nq, dev)
        uniform = not isinstance(k, torch.Tensor) and np.ndim(k) == 0
        uk = int(kw.get("uniform_k", 0))  # rows of uk slots whatever k[] holds
        if out is None:  # (with `out` given nothing here waits on the device)
            total = uk * nq if uk else int(k) * nq if uniform else int(kt.clamp(0, B.MAX_K).sum().item())
            ids = torch.empty(total, dtype=torch.int32, device=dev)
            dists = torch.empty(total, dtype=torch.float32, device=dev)
        else:
            ids, dists = out
        st = torch.empty((nq, 2), dtype=torch.int32, device=dev) if stats else None
        p = self.params(**kw)
        if uniform and p.max_k == 0:
            p.max_k = int(k)
        if uniform and "uniform_k" not in kw and p.max_k == int(k):
            p.uniform_k = int(k)  # one k for the batch: outputs at i * k, no planning kernel
        if not isinstance(ef, torch.Tensor) and np.ndim(ef) == 0 and p.max_ef == 0:
            p.max_ef = int(ef)
        ws_ptr, ws_bytes = (workspace.data_ptr(), workspace.numel() * workspace.element_size()) \
            if workspace is not None else (None, 0)
        rc = B.lib().sqg_search_ex(self._h, queries.data_ptr(), nq, kt.data_ptr(), et.data_ptr(), ids.data_ptr(),
                                   dists.data_ptr(), C.byref(p), ws_ptr, ws_bytes,
                                   st.data_ptr() if st is not None else None, _stream_ptr(stream))
        B.check(rc, "sqg_search_ex")
        if uniform or uk:
            ids, dists = ids.view(nq, uk or int(k)), dists.view(nq, uk or int(k))
        return (ids, dists, st) if stats else (ids, dists)

    def search_plain(self, queries: torch.Tensor, k: torch.Tensor, ef: torch.Tensor, out_ids: torch.Tensor,
                     out_dists: torch.Tensor, stream=None) -> None:
        """sqg_search exactly as the C ABI gives it (device k[], ef[])."""
        rc = B.lib().sqg_search(self._h, queries.data_ptr(), queries.shape[0], k.data_ptr(), ef.data_ptr(),
                                out_ids.data_ptr(), out_dists.data_ptr(), _stream_ptr(stream))
        B.check(rc, "sqg_search")

    def search_trace(self, queries: torch.Tensor, k: int, ef: int, gt: torch.Tensor | None, trace_cap: int,
                     stream=None, path_cap: int = 0, **kw):
        """Search that records the learned stop's features (and hits against
        gt) at every evaluation point, and/or the expansion order.  Returns
        ids, dists, stats, feats (nq, cap, 16), hits (nq, cap), counts (nq,)
        and, with path_cap > 0, path (nq, path_cap; -1 past the last hop)."""
        queries = self.fit_queries(queries)
        nq, dev = queries.shape[0], queries.device
        kt, et = _i32(k, nq, dev), _i32(ef, nq, dev)
        ids = torch.empty(nq * k, dtype=torch.int32, device=dev)
        dists = torch.empty(nq * k, dtype=torch.float32, device=dev)
        st = torch.empty((nq, 2), dtype=torch.int32, device=dev)
        feats = hits = cnt = None
        if trace_cap > 0:
            feats = torch.zeros((nq, trace_cap, B.MLP_IN), dtype=torch.float32, device=dev)
            hits = torch.full((nq, trace_cap), -1, dtype=torch.int32, device=dev)
            cnt = torch.zeros(nq, dtype=torch.int32, device=dev)
        path = torch.full((nq, path_cap), -1, dtype=torch.int32, device=dev) if path_cap > 0 else None
        p = self.params(max_k=k, max_ef=ef, **kw)
        gtp, gtk = (gt.data_ptr(), gt.shape[1]) if gt is not None else (None, 0)
        ptr = lambda t: t.data_ptr() if t is not None else None  # noqa: E731
        rc = B.lib().sqg_search_trace(self._h, queries.contiguous().data_ptr(), nq, kt.data_ptr(), et.data_ptr(),
                                      ids.data_ptr(), dists.data_ptr(), C.byref(p), st.data_ptr(), gtp, gtk,
                                      ptr(feats), ptr(hits), ptr(cnt), trace_cap, ptr(path), path_cap,
                                      _stream_ptr(stream))
        B.check(rc, "sqg_search_trace")
        out = (ids.view(nq, k), dists.view(nq, k), st, feats, hits, cnt)
        return out + (path,) if path_cap > 0 else out

    def workspace_size(self, nq: int, max_k: int, max_ef: int, **kw) -> int:
        """Workspace bytes for a batch; keyword arguments are search
        parameters (the tuning knobs change the size)."""
        if kw:
            p = self.params(**{a: b for a, b in kw.items() if a not in ("max_k", "max_ef")})
            n = B.lib().sqg_workspace_size_ex(self._h, nq, max_k, max_ef, C.byref(p))
        else:
            n = B.lib().sqg_workspace_size(self._h, nq, max_k, max_ef)
        if n == 0:
            raise B.SqgError(-1, "sqg_workspace_size")
        return int(n)

    def search_host(self, queries: np.ndarray, k: int, ef: int, *, pinned: tuple | None = None, **kw):
        """End-to-end search from HOST arrays: copy the queries in, search,
        copy (ids, dists) back; returns numpy arrays."""
        nq = queries.shape[0]
        dev = torch.device("cuda", self.device)
        if pinned is None:
            qh = torch.from_numpy(np.ascontiguousarray(queries, dtype=np.float32)).pin_memory()
            ih = torch.empty((nq, k), dtype=torch.int32).pin_memory()
            dh = torch.empty((nq, k), dtype=torch.float32).pin_memory()
        else:
            qh, ih, dh = pinned
        qd = qh.to(dev, non_blocking=True)
        ids, dists = self.search(qd, k, ef, **kw)
        ih.copy_(ids, non_blocking=True)
        dh.copy_(dists, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return ih.numpy(), dh.numpy()

    def host_pipeline(self, nq: int, k: int, ef: int, depth: int = 2, **kw) -> "HostPipeline":
        """A pipelined end-to-end search over host batches of nq queries."""
        return HostPipeline(self, nq, k, ef, depth=depth, **kw)

    # ------------------------------------------------------------------ test hooks
    def prepare_queries(self, queries: torch.Tensor, stream=None):
        queries = self.fit_queries(queries)
        nq = queries.shape[0]
        dev = queries.device
        qrot = torch.empty((nq, self.d), dtype=torch.float32, device=dev)
        planes = torch.empty((nq, 4, self.d // 32), dtype=torch.int32, device=dev)
        scal = torch.empty((nq, 4), dtype=torch.float32, device=dev)
        B.check(B.lib().sqg_prepare_queries(self._h, queries.contiguous().data_ptr(), nq, qrot.data_ptr(),
                                            planes.data_ptr(), scal.data_ptr(), _stream_ptr(stream)),
                "sqg_prepare_queries")
        return qrot, planes, scal

    def prepare_queries_tc(self, queries: torch.Tensor, stream=None):
        """The tensor-core rotation and the exact quantization after it.

        Returns (q' from the tensor cores, planes, scalars, coordinates the
        exact pass recomputed); planes and scalars equal prepare_queries'."""
        nq = queries.shape[0]
        dev = queries.device
        qrot = torch.empty((nq, self.d), dtype=torch.float32, device=dev)
        planes = torch.empty((nq, 4, self.d // 32), dtype=torch.int32, device=dev)
        scal = torch.empty((nq, 4), dtype=torch.float32, device=dev)
        rec = torch.zeros(1, dtype=torch.int32, device=dev)
        B.check(B.lib().sqg_prepare_queries_tc(self._h, queries.contiguous().data_ptr(), nq, qrot.data_ptr(),
                                               planes.data_ptr(), scal.data_ptr(), rec.data_ptr(),
                                               _stream_ptr(stream)), "sqg_prepare_queries_tc")
        return qrot, planes, scal, rec

    def estimate_block(self, queries: torch.Tensor, v: torch.Tensor, eps0: float = 0.0, stream=None):
        queries = self.fit_queries(queries)
        nq, dev, R = queries.shape[0], queries.device, self.degree
        S = torch.empty((nq, R), dtype=torch.int32, device=dev)
        est = torch.empty((nq, R), dtype=torch.float32, device=dev)
        key = torch.empty((nq, R), dtype=torch.float32, device=dev)
        dc = torch.empty(nq, dtype=torch.float32, device=dev)
        vv = v.to(device=dev, dtype=torch.int32).contiguous()
        B.check(B.lib().sqg_estimate_block(self._h, queries.contiguous().data_ptr(), nq, vv.data_ptr(), eps0,
                                           S.data_ptr(), est.data_ptr(), key.data_ptr(), dc.data_ptr(),
                                           _stream_ptr(stream)), "sqg_estimate_block")
        return S, est, key, dc

    def status(self, stream=None) -> int:
        s = C.c_uint32()
        B.check(B.lib().sqg_get_status(self._h, _stream_ptr(stream), C.byref(s)), "sqg_get_status")
        return int(s.value)


class HostPipeline:
    """End-to-end search over a sequence of host batches of one shape: batch
    i is copied in from pinned host memory, searched and its (ids, dists)
    copied back on stream i % depth, so one batch's copies overlap another's
    search.  Each slot owns its device buffers, workspace and pinned result
    buffers, and replays one CUDA graph of its search and result copies (the
    search's host-side launch costs about 30 us of Python and driver time,
    the replay a few); only the copy in from the caller's tensor is issued
    per batch.  Nothing allocates or waits on the device inside submit()
    except for the slot being reused.

        pipe = ix.host_pipeline(nq, k, ef)
        for qh in pinned_batches:        # (nq, d) float32, pinned
            done = pipe.submit(qh)       # results of an earlier batch, or None
        rest = pipe.drain()              # the remaining results, in order
    """

    class _Slot:
        pass

    def __init__(self, ix: Index, nq: int, k: int, ef: int, depth: int = 2, **kw):
        if depth < 1:
            raise ValueError("depth must be >= 1")
        self.ix, self.nq, self.k, self.ef, self.kw = ix, int(nq), int(k), int(ef), dict(kw)
        dev = torch.device("cuda", ix.device)
        ws_bytes = ix.workspace_size(nq, k, ef, **kw)
        self.slots, self.order, self.count = [], [], 0
        for _ in range(depth):
            sl = HostPipeline._Slot()
            sl.stream = torch.cuda.Stream(device=dev)
            sl.qd = torch.empty((nq, ix.d), dtype=torch.float32, device=dev)
            sl.kt = torch.full((nq,), self.k, dtype=torch.int32, device=dev)
            sl.et = torch.full((nq,), self.ef, dtype=torch.int32, device=dev)
            sl.ids = torch.empty(nq * self.k, dtype=torch.int32, device=dev)
            sl.dists = torch.empty(nq * self.k, dtype=torch.float32, device=dev)
            sl.ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
            sl.ih = torch.empty((nq, self.k), dtype=torch.int32).pin_memory()
            sl.dh = torch.empty((nq, self.k), dtype=torch.float32).pin_memory()
            sl.event = torch.cuda.Event()
            sl.busy = False
            sl.qd.zero_()
            with torch.cuda.stream(sl.stream):  # warm-up outside the capture
                self._search(sl, sl.stream)
            torch.cuda.synchronize(dev)
            sl.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(sl.graph, stream=sl.stream):
                self._search(sl, sl.stream)
            self.slots.append(sl)
        torch.cuda.synchronize(dev)

    def _search(self, sl, stream):
        """The slot's search of sl.qd and the copies of its results into the
        slot's pinned buffers, on `stream` (captured once per slot)."""
        self.ix.search(sl.qd, sl.kt, sl.et, out=(sl.ids, sl.dists), workspace=sl.ws, stream=stream,
                       max_k=self.k, max_ef=self.ef, uniform_k=self.k, **self.kw)
        sl.ih.copy_(sl.ids.view(self.nq, self.k), non_blocking=True)
        sl.dh.copy_(sl.dists.view(self.nq, self.k), non_blocking=True)

    def _collect(self, sl):
        sl.event.synchronize()
        sl.busy = False
        return sl.ih.numpy().copy(), sl.dh.numpy().copy()

    def submit(self, qh: torch.Tensor):
        """Start one batch (a pinned (nq, d) float32 host tensor, left
        untouched until its results come back); returns the (ids, dists) of
        the batch submitted `depth` calls earlier, or None."""
        if qh.shape != (self.nq, self.ix.d) or qh.dtype != torch.float32 or qh.is_cuda:
            raise ValueError(f"expected a host float32 tensor of shape ({self.nq}, {self.ix.d})")
        sl = self.slots[self.count % len(self.slots)]
        done = self._collect(sl) if sl.busy else None
        with torch.cuda.stream(sl.stream):
            sl.qd.copy_(qh, non_blocking=True)
            sl.graph.replay()
            sl.event.record(sl.stream)
        sl.busy = True
        self.count += 1
        return done

    def drain(self) -> list:
        """The results of every batch still in flight, oldest first."""
        out = []
        n = len(self.slots)
        for j in range(n):
            sl = self.slots[(self.count + j) % n]
            if sl.busy:
                out.append(self._collect(sl))
        return out


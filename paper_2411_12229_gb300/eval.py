"""Accuracy metrics of Sec. 5.1: recall |G cap S|/K and the average distance
ratio, with exact ground truth.

Ground truth takes candidates from a GPU matrix product (library GEMM) when
a device is given, then re-ranks them exactly in fp64 on the host with ties
broken by id; with no device it is plain fp64 brute force on the host.
"""

from __future__ import annotations

import numpy as np


def _exact_rerank(base: np.ndarray, q: np.ndarray, cand: np.ndarray, k: int):
    ids = np.empty((q.shape[0], k), dtype=np.int64)
    dd = np.empty((q.shape[0], k), dtype=np.float64)
    for i in range(q.shape[0]):
        c = np.unique(cand[i])
        diff = base[c].astype(np.float64) - q[i].astype(np.float64)
        dist = np.einsum("ij,ij->i", diff, diff)
        o = np.lexsort((c, dist))[:k]
        ids[i], dd[i] = c[o], dist[o]
    return ids, dd


def ground_truth(base: np.ndarray, queries: np.ndarray, k: int, device=None, margin: int = 32,
                 chunk: int = 1 << 18, qchunk: int = 8192):
    """Exact k nearest neighbours (ids int64, squared distances fp64).  On a
    device the queries go through in chunks of `qchunk` rows, so the
    candidate matrix stays at qchunk x chunk floats."""
    if device is not None and queries.shape[0] > qchunk:
        parts = [ground_truth(base, queries[a:a + qchunk], k, device, margin, chunk, qchunk)
                 for a in range(0, queries.shape[0], qchunk)]
        return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])
    base = np.ascontiguousarray(base, dtype=np.float32)
    queries = np.ascontiguousarray(queries, dtype=np.float32)
    kc = min(base.shape[0], k + margin)
    if device is None:
        cand = np.empty((queries.shape[0], kc), dtype=np.int64)
        bn = np.einsum("ij,ij->i", base.astype(np.float64), base.astype(np.float64))
        for a in range(0, queries.shape[0], 256):
            qq = queries[a:a + 256].astype(np.float64)
            d = bn[None, :] - 2.0 * qq @ base.T.astype(np.float64)
            cand[a:a + 256] = np.argpartition(d, kc - 1, axis=1)[:, :kc]
        return _exact_rerank(base, queries, cand, k)
    import torch
    dev = torch.device("cuda", device) if isinstance(device, int) else device
    qd = torch.from_numpy(queries).to(dev)
    best_d = torch.full((queries.shape[0], kc), float("inf"), device=dev)
    best_i = torch.zeros((queries.shape[0], kc), dtype=torch.int64, device=dev)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for a in range(0, base.shape[0], chunk):
            b = torch.from_numpy(base[a:a + chunk]).to(dev)
            d = (b * b).sum(1)[None, :] - 2.0 * (qd @ b.T)
            v, i = torch.topk(d, min(kc, d.shape[1]), dim=1, largest=False)
            allv = torch.cat([best_d, v], 1)
            alli = torch.cat([best_i, i + a], 1)
            o = torch.topk(allv, kc, dim=1, largest=False).indices
            best_d, best_i = torch.gather(allv, 1, o), torch.gather(alli, 1, o)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return _exact_rerank(base, queries, best_i.cpu().numpy(), k)


def recall(ids: np.ndarray, gt: np.ndarray, k: int) -> float:
    """Mean |G cap S| / K over queries (Sec. 5.1)."""
    ids = np.asarray(ids)[:, :k].astype(np.int64)
    gt = np.asarray(gt)[:, :k].astype(np.int64)
    hit = [len(np.intersect1d(ids[i][ids[i] >= 0], gt[i])) for i in range(gt.shape[0])]
    return float(np.mean(hit)) / k


def recall_per_query(ids, gt, k) -> np.ndarray:
    ids = np.asarray(ids)[:, :k].astype(np.int64)
    gt = np.asarray(gt)[:, :k].astype(np.int64)
    return np.array([len(np.intersect1d(ids[i][ids[i] >= 0], gt[i])) / k for i in range(gt.shape[0])])


def average_distance_ratio(dists: np.ndarray, gt_dists: np.ndarray, k: int) -> float:
    """Mean over queries and ranks of ||o_i - q|| / ||o*_i - q|| (Sec. 5.1);
    inputs are squared distances, ranks with a zero true distance skipped."""
    d = np.sqrt(np.asarray(dists, dtype=np.float64)[:, :k])
    g = np.sqrt(np.asarray(gt_dists, dtype=np.float64)[:, :k])
    ok = (g > 0) & np.isfinite(d)
    return float(np.mean(d[ok] / g[ok]))

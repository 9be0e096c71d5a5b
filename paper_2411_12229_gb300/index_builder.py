"""Index construction driver (Algorithm 2, Indexing, Sec. 3.2).

The paper builds the graph by starting from a random R-regular graph and
repeating, t times: prepare the FastScan data (quantize every edge), search
the current graph for candidates of every vertex with its own query
algorithm, prune the candidates with NSG's rule, adjust the graph; then
supplement edges so that every vertex has exactly R, and prepare the final
FastScan data.  Here:

* the FastScan data and the file are written by ``sqg_write_index`` (host);
* the candidate search of every vertex is the GPU search kernel itself
  (``Index.search`` with the vertex's own vector as the query, k = L results
  by exact distance), which is the paper's "leverage our search to
  accelerate index construction";
* pruning, reverse edges and the adaptive-angle supplement run in
  ``sqg_build_graph`` (host, multithreaded), so every intermediate graph
  already has exactly R edges and can be searched by the same kernel;
* without a GPU (tests) the candidates come from a brute-force kNN.
"""

from __future__ import annotations

import ctypes as C
import os
import pathlib
import time

import numpy as np

from . import _binding as B


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def random_rotation(d: int, seed: int) -> np.ndarray:
    """P^-1 of a Haar-random orthogonal P (Sec. 2.2, the JLT of Eq. (3)):
    QR of a seeded standard Gaussian matrix, column signs fixed by diag(R),
    in fp64; returned as float32 row-major."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(entropy=seed, spawn_key=(11, d))))
    a = g.standard_normal((d, d))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    return np.ascontiguousarray(q.T, dtype=np.float32)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 (Steele, Lea, Flood 2014): the output for each state x (uint64)."""
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def fjlt_signs(d: int, seed: int) -> np.ndarray:
    """3 x d signs of the fast JLT: -1 where bit 63 of
    splitmix64(seed ^ (r << 32 | i)) is set."""
    r = np.arange(3, dtype=np.uint64)[:, None]
    i = np.arange(d, dtype=np.uint64)[None, :]
    x = np.uint64(seed) ^ ((r << np.uint64(32)) | i)
    return np.where(splitmix64(x) >> np.uint64(63), -1.0, 1.0)


def fjlt_matrix(d: int, seed: int) -> np.ndarray:
    """The fast JLT (Sec. 3.1.4) as a dense matrix, fp64 -> float32: rows of
    c H S_3 c H S_2 c H S_1 with H the Walsh-Hadamard matrix (Sylvester
    order) and c = 1/sqrt(d); d a power of 2."""
    if d & (d - 1):
        raise ValueError("the fast JLT needs d a power of 2")
    h = np.ones((1, 1))
    while h.shape[0] < d:
        h = np.block([[h, h], [h, -h]])
    s = fjlt_signs(d, seed)
    m = np.eye(d)
    for r in range(3):
        m = (h @ (s[r][:, None] * m)) / np.sqrt(d)
    return np.ascontiguousarray(m, dtype=np.float32)


def knn_host(data: np.ndarray, k: int, threads: int = 0) -> np.ndarray:
    data = np.ascontiguousarray(data, dtype=np.float32)
    out = np.empty((data.shape[0], k), dtype=np.uint32)
    B.check(B.lib().sqg_knn_host(_p(data), data.shape[0], data.shape[1], k, _p(out), threads), "sqg_knn_host")
    return out


def medoid(data: np.ndarray, threads: int = 0) -> int:
    data = np.ascontiguousarray(data, dtype=np.float32)
    return int(B.lib().sqg_medoid(_p(data), data.shape[0], data.shape[1], threads))


def build_graph(data: np.ndarray, cand: np.ndarray, R: int, entry: int, seed: int = 3,
                threads: int = 0, device: int | None = None, regular: bool = True) -> tuple[np.ndarray, dict]:
    """Algorithm 2's adjust step: prune, reverse edges, angle rule, random
    fill, reachability (Sec. 3.2).  device=None: on the host threads; a
    device: the per-vertex steps on that GPU (the same rows bit for bit).
    regular=False: the degree-unaligned graph of the "w/o GR" ablation
    (Sec. 5): no angle rule, no random fill, unused slots NO_ID."""
    data = np.ascontiguousarray(data, dtype=np.float32)
    cand = np.ascontiguousarray(cand, dtype=np.uint32)
    n = data.shape[0]
    adj = np.empty((n, R), dtype=np.uint32)
    st = np.zeros(5, dtype=np.uint64)
    if device is not None and (cand.shape[1] > 512 or min(R, n - 1) > 64):
        device = None  # longer lists than the GPU kernels keep: the host builds it
    flags = 0 if regular else B.GRAPH_IRREGULAR
    if device is None and regular:
        B.check(B.lib().sqg_build_graph(_p(data), n, data.shape[1], _p(cand), cand.shape[1], R, entry, seed,
                                        _p(adj), _p(st), threads), "sqg_build_graph")
    else:
        B.check(B.lib().sqg_build_graph_ex(_p(data), n, data.shape[1], _p(cand), cand.shape[1], R, entry, seed,
                                           flags, _p(adj), _p(st), threads, -1 if device is None else int(device)),
                "sqg_build_graph_ex")
    out = dict(avg_nsg_degree=st[0] / 1000.0, supplemented=int(st[1]), random_filled=int(st[2]),
               repairs=int(st[3]))
    if device is not None:
        out["host_refined"] = int(st[4])
    return adj, out


def unit_rows(data: np.ndarray, chunk: int = 1 << 16) -> np.ndarray:
    """Each row scaled to unit norm (norm in fp64; zero rows stay zero):
    the vectors of a cosine index."""
    out = np.empty(data.shape, np.float32)
    for a in range(0, data.shape[0], chunk):
        x = data[a:a + chunk].astype(np.float64)
        nrm = np.sqrt((x * x).sum(axis=1, keepdims=True))
        out[a:a + chunk] = np.where(nrm > 0, x / np.where(nrm > 0, nrm, 1.0), 0.0)
    return out


def write_index(path, data: np.ndarray, adj: np.ndarray, rot: np.ndarray, entry: int, seed_rotation: int,
                seed_graph: int, threads: int = 0, rotation_kind: int = 0, metric: int = 0) -> None:
    data = np.ascontiguousarray(data, dtype=np.float32)
    adj = np.ascontiguousarray(adj, dtype=np.uint32)
    rot = np.ascontiguousarray(rot, dtype=np.float32)
    B.check(B.lib().sqg_write_index2(str(path).encode(), _p(data), data.shape[0], data.shape[1], _p(adj),
                                     adj.shape[1], _p(rot), entry, seed_rotation, seed_graph, threads, rotation_kind,
                                     metric),
            f"sqg_write_index2({path})")


def random_graph(n: int, R: int, seed: int) -> np.ndarray:
    """R distinct random out-neighbours per vertex, none the vertex itself
    (the random initial graph of Algorithm 2)."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(entropy=seed, spawn_key=(12,))))
    if n - 1 < R:
        raise ValueError("need n > R")
    adj = g.integers(0, n - 1, size=(n, R), dtype=np.int64)
    adj += adj >= np.arange(n)[:, None]  # skip the vertex itself
    for _ in range(64):
        s = np.sort(adj, axis=1)
        bad = np.nonzero((s[:, 1:] == s[:, :-1]).any(axis=1))[0]
        if bad.size == 0:
            break
        for u in bad:
            row = g.choice(n - 1, size=R, replace=False)
            row = row + (row >= u)
            adj[u] = row
    return adj.astype(np.uint32)


def build_index(path, data: np.ndarray, R: int, *, iterations: int | None = None, ef_build: int = 128,
                cand_k: int | None = None, path_cand: int | None = None, rot_seed: int = 2, graph_seed: int = 3,
                device: int | None = None, init: str = "auto", threads: int = 0, rotation: str = "dense",
                metric: str = "l2", regular: bool = True, log=None) -> dict:
    """Build an index file at `path` from base vectors `data` (n x d).

    device=None: host-only build from an exact kNN (small n).
    device given: Algorithm 2 with the GPU search providing the candidates
    of every vertex: the cand_k nearest vertices the search expanded plus
    the first path_cand vertices on its path from the entry point (as NSG
    takes the visited set, so that long edges between regions survive the
    pruning); init "random" (the paper) or "knn" (host brute force).

    rotation "dense": a Haar-random P^-1 (stored, applied as a d x d
    product); "fjlt": the fast JLT of Sec. 3.1.4, the data zero-padded to
    the next power of 2 (queries are padded the same way by the API).

    regular=False builds the degree-unaligned graph of the "w/o GR"
    ablation (Sec. 5) in every iteration: rows keep their pruned edges and
    end in NO_ID slots.

    metric "l2": squared Euclidean; "cosine": cosine similarity as
    Euclidean search between unit vectors -- the data are scaled to unit
    norm here, the library scales every query (Sec. 3 names both metrics)."""
    t0 = time.time()
    data = np.ascontiguousarray(data, dtype=np.float32)
    if metric not in ("l2", "cosine"):
        raise ValueError("metric is 'l2' or 'cosine'")
    mcode = 1 if metric == "cosine" else 0
    if mcode:
        data = unit_rows(data)
    if rotation == "fjlt":
        dp = 1 << max(5, int(np.ceil(np.log2(data.shape[1]))))
        if dp != data.shape[1]:
            data = np.ascontiguousarray(np.pad(data, ((0, 0), (0, dp - data.shape[1]))))
    elif rotation != "dense":
        raise ValueError("rotation is 'dense' or 'fjlt'")
    kind = 1 if rotation == "fjlt" else 0
    n, d = data.shape
    if n <= R:  # every vertex needs R distinct neighbours other than itself
        raise ValueError(f"an index of degree {R} needs more than {R} vectors (got {n})")
    cand_k = cand_k or 2 * R
    rot = fjlt_matrix(d, rot_seed) if kind else random_rotation(d, rot_seed)
    entry = medoid(data, threads)
    info = dict(n=n, d=d, R=R, entry=entry, iterations=[])
    tmp = pathlib.Path(str(path) + ".tmp")
    if init == "auto":
        init = "knn" if (device is None or n <= 50_000) else "random"
    if init == "knn":
        cand = knn_host(data, min(cand_k, n - 1), threads)
        adj, st = build_graph(data, cand, R, entry, graph_seed, threads, device, regular)
        info["iterations"].append(dict(source="knn", **st))
    else:
        adj = random_graph(n, R, graph_seed)
    if iterations is None:
        iterations = 0 if device is None else (3 if init == "random" else 1)
    write_index(tmp if iterations else path, data, adj, rot, entry, rot_seed, graph_seed, threads, kind, mcode)
    if iterations:
        import torch

        from .api import Index
        dev = torch.device("cuda", device)
        xd = torch.from_numpy(data).to(dev)
        k_res = min(cand_k, n)
        pc = R if path_cand is None else path_cand
        for it in range(iterations):
            t1 = time.time()
            ix = Index(tmp, device)
            cand = np.empty((n, k_res + pc), dtype=np.uint32)
            step = 1 << 18
            with torch.cuda.device(dev):
                for a in range(0, n, step):
                    b = min(n, a + step)
                    if pc > 0:
                        r = ix.search_trace(xd[a:b], k_res, max(ef_build, k_res), None, 0, path_cap=pc)
                        cand[a:b] = torch.cat([r[0], r[-1]], 1).cpu().numpy().view(np.uint32)
                    else:
                        ids, _ = ix.search(xd[a:b], k_res, max(ef_build, k_res))
                        cand[a:b] = ids.cpu().numpy().view(np.uint32)
            ix.close()
            t2 = time.time()
            adj, st = build_graph(data, cand, R, entry, graph_seed + it + 1, threads, device, regular)
            t3 = time.time()
            final = it == iterations - 1
            write_index(path if final else tmp, data, adj, rot, entry, rot_seed, graph_seed, threads, kind, mcode)
            st.update(search_s=round(t2 - t1, 2), graph_s=round(t3 - t2, 2), write_s=round(time.time() - t3, 2))
            info["iterations"].append(dict(source="gpu-search", seconds=time.time() - t1, **st))
            if log:
                log(f"build iteration {it + 1}/{iterations}: {time.time() - t1:.1f}s {st}")
        if tmp.exists():
            os.remove(tmp)
    info["seconds"] = time.time() - t0
    return info

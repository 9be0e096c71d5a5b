"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws vectors and nothing else: it holds none of the search
method's arithmetic (no rotation, no quantization, no distance estimate), so
that the CUDA path and the CPU oracle can both take their inputs from it.

The paper evaluates on real datasets (Sec. 5.1, Table "Statistics of the
datasets": SIFT 1M x 128, GIST 1M x 960, Deep-100M 96-d cosine, ...).  Those
are replaced here by isotropic Gaussian mixtures with the same N, D and query
counts:

* centres ~ N(0, 4 I), per-point noise sigma = 1, uniform mixture weights;
* ``dim_scale="loguniform"``: every coordinate i is multiplied by
  s_i = exp(U[ln 0.1, ln 10]), one draw per dimension shared by base and
  query vectors (SIFT-like uneven per-dimension scales);
* ``dim_scale="power"``: coordinate i (1-based) is multiplied by i^(-1/4),
  so its variance decays as 1/sqrt(i), then the absolute value is taken
  (GIST-like non-negative data);
* ``unit_norm``: every vector is projected onto the unit sphere
  (cosine-style data, Sec. 3 "only supports ... Euclidean space and cosine
  similarity").

Every draw comes from numpy's PCG64 keyed by (seed, stream, chunk), so any
row range can be regenerated on its own and the same rows come out on every
machine.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

_CHUNK = 65536  # rows per independently seeded chunk

# stream identifiers (spawn keys of the SeedSequence)
_S_CENTERS, _S_SCALE, _S_BASE, _S_QUERY, _S_TRAIN, _S_PARAMS, _S_ARRIVALS = range(7)


@dataclasses.dataclass(frozen=True)
class Workload:
    """A synthetic workload: dataset shape, mixture recipe and search knobs."""

    name: str
    n: int                 # base vectors
    d: int                 # dimension (a multiple of 32)
    n_components: int      # Gaussian mixture components
    n_queries: int         # test queries
    degree: int            # graph out-degree R (a multiple of 32)
    k: int = 10
    ef: tuple = (32, 64, 128)
    n_train: int = 0       # training queries (learned early stop)
    dim_scale: str = "none"  # "none" | "loguniform" | "power"
    unit_norm: bool = False
    center_std: float = 2.0
    noise_std: float = 1.0
    seed: int = 0
    mixed_k: tuple = ()    # per-query k drawn uniformly from this set
    ef_factor_max: int = 0  # per-query ef drawn uniformly in [k, ef_factor_max*k]

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


EF_SWEEP = (16, 24, 32, 36, 40, 44, 48, 56, 64, 80, 96, 112, 128, 160, 192, 256, 320, 384, 512)

# The five workloads, named by what they are.
TINY_10K_D128 = Workload("tiny-10k-d128", 10_000, 128, 64, 200, 32, ef=(32, 64, 128))
BATCHED_1M_D128 = Workload("batched-1m-d128", 1_000_000, 128, 1024, 10_000, 32,
                           ef=EF_SWEEP, dim_scale="loguniform")
HIGHDIM_1M_D960 = Workload("highdim-1m-d960", 1_000_000, 960, 512, 10_000, 64,
                           ef=EF_SWEEP, n_train=50_000, dim_scale="power")
UNEVEN_1M_D1536 = Workload("uneven-1m-d1536", 1_000_000, 1536, 2048, 20_000, 32,
                           unit_norm=True, mixed_k=(1, 10, 100), ef_factor_max=8)
SERVING_4M_D96 = Workload("serving-4m-d96", 4_000_000, 96, 4096, 10_000, 32,
                          ef=EF_SWEEP, mixed_k=(10, 100))

WORKLOADS = {w.name: w for w in (TINY_10K_D128, BATCHED_1M_D128, HIGHDIM_1M_D960,
                                  UNEVEN_1M_D1536, SERVING_4M_D96)}


def _rng(w: Workload, stream: int, chunk: int = 0) -> np.random.Generator:
    ss = np.random.SeedSequence(entropy=w.seed, spawn_key=(stream, chunk))
    return np.random.Generator(np.random.PCG64(ss))


def centers(w: Workload) -> np.ndarray:
    """Mixture centres, (n_components, d) float32, ~ N(0, center_std^2 I)."""
    g = _rng(w, _S_CENTERS)
    return (g.standard_normal((w.n_components, w.d), dtype=np.float32)
            * np.float32(w.center_std))


def dim_scales(w: Workload) -> np.ndarray | None:
    """Per-dimension multipliers shared by base and query vectors (or None)."""
    if w.dim_scale == "none":
        return None
    if w.dim_scale == "loguniform":
        g = _rng(w, _S_SCALE)
        u = g.uniform(math.log(0.1), math.log(10.0), size=w.d)
        return np.exp(u).astype(np.float32)
    if w.dim_scale == "power":
        i = np.arange(1, w.d + 1, dtype=np.float64)
        return (i ** -0.25).astype(np.float32)
    raise ValueError(f"unknown dim_scale {w.dim_scale!r}")


def _draw(w: Workload, stream: int, lo: int, hi: int, C: np.ndarray,
          scale: np.ndarray | None) -> np.ndarray:
    out = np.empty((hi - lo, w.d), dtype=np.float32)
    c0 = lo // _CHUNK
    c1 = (hi - 1) // _CHUNK if hi > lo else c0 - 1
    for c in range(c0, c1 + 1):
        r0, r1 = c * _CHUNK, (c + 1) * _CHUNK
        g = _rng(w, stream, c)
        comp = g.integers(0, w.n_components, size=_CHUNK)
        a, b = max(lo, r0), min(hi, r1)
        # the stream is sequential: rows past b are never needed
        x = g.standard_normal((b - r0, w.d), dtype=np.float32)
        sel = slice(a - r0, b - r0)
        xs = x[sel]
        xs *= np.float32(w.noise_std)
        xs += C[comp[sel]]
        if scale is not None:
            xs *= scale
        if w.dim_scale == "power":
            np.abs(xs, out=xs)
        if w.unit_norm:
            nrm = np.sqrt(np.einsum("ij,ij->i", xs.astype(np.float64), xs.astype(np.float64)))
            nrm[nrm == 0] = 1.0
            xs /= nrm[:, None].astype(np.float32)
        out[a - lo:b - lo] = xs
    return out


def base(w: Workload, lo: int = 0, hi: int | None = None) -> np.ndarray:
    """Rows [lo, hi) of the base set, float32 (hi - lo, d)."""
    hi = w.n if hi is None else hi
    if not (0 <= lo <= hi <= w.n):
        raise ValueError("row range out of bounds")
    return _draw(w, _S_BASE, lo, hi, centers(w), dim_scales(w))


def queries(w: Workload, n: int | None = None) -> np.ndarray:
    """The first n test queries (default: all), float32 (n, d)."""
    n = w.n_queries if n is None else n
    return _draw(w, _S_QUERY, 0, n, centers(w), dim_scales(w))


def train_queries(w: Workload, n: int | None = None) -> np.ndarray:
    """Training queries for the learned early stop, float32 (n, d)."""
    n = w.n_train if n is None else n
    return _draw(w, _S_TRAIN, 0, n, centers(w), dim_scales(w))


def query_k_ef(w: Workload, n: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Per-query (k, ef) for mixed batches: k ~ U(mixed_k), ef ~ U[k, f*k]."""
    n = w.n_queries if n is None else n
    g = _rng(w, _S_PARAMS)
    ks = np.asarray(w.mixed_k, dtype=np.int32)
    k = ks[g.integers(0, len(ks), size=n)]
    f = max(1, w.ef_factor_max)
    ef = g.integers(k, f * k + 1).astype(np.int32)
    return k.astype(np.int32), ef


def poisson_arrivals(rate_qps: float, n: int, seed: int = 5) -> np.ndarray:
    """Arrival times (seconds, float64, increasing) of a Poisson process."""
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(
        entropy=seed, spawn_key=(_S_ARRIVALS, int(rate_qps)))))
    return np.cumsum(g.exponential(1.0 / rate_qps, size=n))


def small(w: Workload, n: int, n_queries: int, n_components: int | None = None) -> Workload:
    """A scaled-down copy of a workload (same recipe, smaller N) for tests."""
    nc = n_components if n_components is not None else max(4, w.n_components * n // w.n)
    return w.with_(name=f"{w.name}-n{n}", n=n, n_queries=n_queries, n_components=nc)

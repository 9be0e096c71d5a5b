"""ctypes binding of the CPU oracle (sqg_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the benchmark's CPU-baseline leg, never by the library.  It shares no
code with the library: the C file has its own index reader, estimator and
search, written from the paper's definitions (see the C file's header for the
equations and algorithm each function follows).
"""

from __future__ import annotations

import ctypes as C
import os
import pathlib
import subprocess
import threading

import numpy as np

HERE = pathlib.Path(__file__).resolve().parent
SRC = HERE / "sqg_oracle.c"
OUT = HERE / "_build" / "liboracle.so"

MLP_IN, MLP_H = 16, 64
MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1  # 5313
STATUS_CAPACITY, STATUS_LEARNED_STOP = 1, 2
NO_ID = 0xFFFFFFFF

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> pathlib.Path:
    """Compile the oracle with gcc (plain C99, no fused multiply-adds other
    than the explicit fmaf calls)."""
    OUT.parent.mkdir(exist_ok=True)
    if force or not OUT.exists() or OUT.stat().st_mtime < SRC.stat().st_mtime:
        tmp = OUT.with_suffix(f".{os.getpid()}.tmp")
        subprocess.run(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                        "-shared", "-o", str(tmp), str(SRC), "-lm"], check=True)
        os.replace(tmp, OUT)
    return OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(str(build()))
            P, U32, U64, I32, F32, F64 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int32, C.c_float, C.c_double
            sig = {
                "orc_index_load": (C.c_int, [C.c_char_p, C.POINTER(P)]),
                "orc_index_free": (None, [P]),
                "orc_index_shape": (None, [P, P, P, P, P, P]),
                "orc_rotation": (P, [P]),
                "orc_metric": (U32, [P]),
                "orc_normalize_f32": (None, [P, U32, P]),
                "orc_raw": (P, [P, U32]),
                "orc_vertex": (None, [P, U32, P, P, P, P, P, P]),
                "orc_rotate_f64": (None, [P, U32, P, P]),
                "orc_rotate_f32": (None, [P, U32, P, P]),
                "orc_splitmix64": (U64, [U64]),
                "orc_fjlt_signs": (None, [U64, U32, P]),
                "orc_fjlt_f64": (None, [P, U32, P, P]),
                "orc_fjlt_f32": (None, [P, U32, P, P]),
                "orc_fjlt_index_signs": (P, [P]),
                "orc_sqdist_f64": (F64, [P, P, U32]),
                "orc_quantize_edge": (None, [P, U32, P, P, P, P]),
                "orc_estimate_unquantized_f64": (None, [P, U32, P, P, P, P]),
                "orc_bruteforce": (None, [P, U64, U32, P, U32, P, P]),
                "orc_quantize_query": (None, [P, U32, P, P, P, P]),
                "orc_exact_dist_f32": (F32, [P, P, U32]),
                "orc_estimate_block": (C.c_int, [P, P, U32, F32, P, P, P, P]),
                "orc_prepare_query": (None, [P, P, P, P, P, P, P]),
                "orc_mlp_logit_f32": (F32, [P, P]),
                "orc_mlp_loss_grad_f64": (F64, [P, P, P, P, C.c_int, P]),
                "orc_adam_step_f64": (None, [P, P, P, P, C.c_int, C.c_int, F64, F64, F64, F64]),
                "orc_adjust_graph": (C.c_int, [P, U64, U32, P, U32, U32, C.c_int, P, P]),
                "orc_search": (C.c_int, [P, P, U32, U32, F32, C.c_int, U32, P, F32, U32, P, P, P,
                                         P, P, P, I32, P, P, U32]),
                "orc_search_record": (C.c_int, [P, P, U32, U32, U32, P, P, P, U32, P, P, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class Index:
    """The oracle's own view of an index file."""

    def __init__(self, path: str | os.PathLike):
        h = C.c_void_p()
        rc = lib().orc_index_load(str(path).encode(), C.byref(h))
        if rc != 0:
            raise OSError(f"oracle: cannot load index {path} (code {rc})")
        self._h = h
        n, d, R, e, bb = C.c_uint64(), C.c_uint32(), C.c_uint32(), C.c_uint32(), C.c_uint32()
        lib().orc_index_shape(h, C.byref(n), C.byref(d), C.byref(R), C.byref(e), C.byref(bb))
        self.n, self.d, self.R, self.entry, self.block_bytes = n.value, d.value, R.value, e.value, bb.value
        self.metric = int(lib().orc_metric(h))  # 0 squared Euclidean, 1 cosine (R16)

    def close(self):
        if self._h:
            lib().orc_index_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rotation(self) -> np.ndarray:
        p = lib().orc_rotation(self._h)
        return np.ctypeslib.as_array(C.cast(p, C.POINTER(C.c_float)), shape=(self.d, self.d)).copy()

    def fjlt_signs(self) -> np.ndarray | None:
        """The fast JLT's 3 x d signs of a version-2 index, else None."""
        p = lib().orc_fjlt_index_signs(self._h)
        if not p:
            return None
        return np.ctypeslib.as_array(C.cast(p, C.POINTER(C.c_float)), shape=(3, self.d)).copy()

    def raw(self, v: int) -> np.ndarray:
        p = lib().orc_raw(self._h, int(v))
        return np.ctypeslib.as_array(C.cast(p, C.POINTER(C.c_float)), shape=(self.d,)).copy()

    def raw_all(self) -> np.ndarray:
        return np.stack([self.raw(v) for v in range(self.n)])

    def vertex(self, v: int) -> dict:
        R, d = self.R, self.d
        ids = np.empty(R, np.uint32)
        bits = np.empty((R, d), np.uint8)
        fa, fr, fe = (np.empty(R, np.float32) for _ in range(3))
        pc = np.empty(R, np.uint32)
        lib().orc_vertex(self._h, int(v), _p(ids), _p(bits), _p(fa), _p(fr), _p(fe), _p(pc))
        return dict(ids=ids, bits=bits, f_add=fa, f_rescale=fr, f_err=fe, popcount=pc)

    def prepare_query(self, q) -> dict:
        q = _f32(q)
        qr = np.empty(self.d, np.float32)
        qbar = np.empty(self.d, np.uint8)
        vl, dl, sq = C.c_float(), C.c_float(), C.c_int32()
        lib().orc_prepare_query(self._h, _p(q), _p(qr), _p(qbar), C.byref(vl), C.byref(dl), C.byref(sq))
        return dict(qrot=qr, qbar=qbar, vl=vl.value, delta=dl.value, sq=sq.value)

    def estimate_block(self, q, v: int, eps0: float = 0.0) -> dict:
        q = _f32(q)
        S = np.empty(self.R, np.int32)
        est, key = np.empty(self.R, np.float32), np.empty(self.R, np.float32)
        dc = C.c_float()
        lib().orc_estimate_block(self._h, _p(q), int(v), eps0, _p(S), _p(est), _p(key), C.byref(dc))
        return dict(S=S, est=est, key=key, dist_c=dc.value)

    def search(self, q, k: int, ef: int, eps0: float = 0.0, multi_estimate: bool = True,
               hop_cap: int | None = None, mlp: np.ndarray | None = None, stop_logit: float = 0.0,
               stop_every: int = 1, gt: np.ndarray | None = None, trace_cap: int = 0, path_cap: int = 0):
        """Algorithm 1 for one query.  Returns (ids, dists, hops, status),
        with trace_cap > 0 also (features, hits), with path_cap > 0 also the
        ids of the first path_cap expanded vertices in order."""
        q = _f32(q)
        ids = np.empty(k, np.uint32)
        dists = np.empty(k, np.float32)
        stats = np.zeros(2, np.uint32)
        cap = default_hop_cap(ef) if hop_cap is None else hop_cap
        mlp_keep = _f32(mlp) if mlp is not None else None
        mp = _p(mlp_keep) if mlp_keep is not None else None
        tf = th = None
        tn = C.c_int32(0)
        if trace_cap > 0:
            tf = np.empty((trace_cap, MLP_IN), np.float32)
            th = np.full(trace_cap, -1, np.int32)
        gtp = np.ascontiguousarray(gt, dtype=np.uint32) if gt is not None else None
        path = np.full(max(path_cap, 1), NO_ID, np.uint32)
        rc = lib().orc_search(self._h, _p(q), k, ef, eps0, int(multi_estimate), cap, mp, stop_logit,
                              stop_every, _p(ids), _p(dists), _p(stats),
                              _p(gtp) if gtp is not None else None,
                              _p(tf) if tf is not None else None, _p(th) if th is not None else None,
                              trace_cap, C.byref(tn), _p(path) if path_cap > 0 else None, path_cap)
        if rc != 0:
            raise ValueError(f"oracle search failed (code {rc})")
        out = [ids, dists, int(stats[0]), int(stats[1])]
        if trace_cap > 0:
            out += [tf[:tn.value], th[:tn.value]]
        if path_cap > 0:
            out.append(path[:min(path_cap, int(stats[0]))])
        return tuple(out)


    def search_record(self, q, k: int, ef: int, hop_cap: int | None = None, rec_cap: int = 64):
        """Algorithm 1 (eps0 = 0, multiple estimates) that also returns the
        beam after each expansion's cut to ef: (ids, dists, hops, status,
        beams), beams[h] = list of (id, key, visited) in beam order."""
        q = _f32(q)
        ids = np.empty(k, np.uint32)
        dists = np.empty(k, np.float32)
        stats = np.zeros(2, np.uint32)
        cap = default_hop_cap(ef) if hop_cap is None else hop_cap
        rm = np.zeros(rec_cap, np.int32)
        ri = np.zeros(rec_cap * ef, np.uint32)
        rk = np.zeros(rec_cap * ef, np.float32)
        rv = np.zeros(rec_cap * ef, np.uint8)
        rc = lib().orc_search_record(self._h, _p(q), k, ef, cap, _p(ids), _p(dists), _p(stats), rec_cap, _p(rm),
                                     _p(ri), _p(rk), _p(rv))
        if rc != 0:
            raise ValueError(f"oracle search failed (code {rc})")
        beams = [[(int(ri[h * ef + i]), float(rk[h * ef + i]), bool(rv[h * ef + i])) for i in range(rm[h])]
                 for h in range(min(rec_cap, int(stats[0])))]
        return ids, dists, int(stats[0]), int(stats[1]), beams


def default_hop_cap(ef: int) -> int:
    """Hop cap used when the caller gives none (a safety bound, R6)."""
    return 4 * int(ef) + 64


def rotate_f64(rot, q) -> np.ndarray:
    rot, q = _f32(rot), _f32(q)
    out = np.empty(rot.shape[0], np.float64)
    lib().orc_rotate_f64(_p(rot), rot.shape[0], _p(q), _p(out))
    return out


def rotate_f32(rot, q) -> np.ndarray:
    rot, q = _f32(rot), _f32(q)
    out = np.empty(rot.shape[0], np.float32)
    lib().orc_rotate_f32(_p(rot), rot.shape[0], _p(q), _p(out))
    return out


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(C.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def fjlt_signs(seed: int, d: int) -> np.ndarray:
    out = np.empty(3 * d, np.float32)
    lib().orc_fjlt_signs(C.c_uint64(seed), d, _p(out))
    return out.reshape(3, d)


def fjlt_f64(signs, q) -> np.ndarray:
    signs, q = _f32(signs), _f32(q)
    out = np.empty(q.shape[0], np.float64)
    lib().orc_fjlt_f64(_p(signs), q.shape[0], _p(q), _p(out))
    return out


def fjlt_f32(signs, q) -> np.ndarray:
    signs, q = _f32(signs), _f32(q)
    out = np.empty(q.shape[0], np.float32)
    lib().orc_fjlt_f32(_p(signs), q.shape[0], _p(q), _p(out))
    return out


def normalize_f32(q) -> np.ndarray:
    """q / ||q|| in fp32 in the order of R16 (a zero query is returned as is)."""
    q = _f32(q)
    out = np.empty(q.shape[0], np.float32)
    lib().orc_normalize_f32(_p(q), q.shape[0], _p(out))
    return out


def quantize_query(qrot) -> dict:
    qrot = _f32(qrot)
    d = qrot.shape[0]
    qbar = np.empty(d, np.uint8)
    vl, dl, sq = C.c_float(), C.c_float(), C.c_int32()
    lib().orc_quantize_query(_p(qrot), d, _p(qbar), C.byref(vl), C.byref(dl), C.byref(sq))
    return dict(qbar=qbar, vl=vl.value, delta=dl.value, sq=sq.value)


def quantize_edge(rot, c, o) -> tuple[np.ndarray, dict]:
    rot, c, o = _f32(rot), _f32(c), _f32(o)
    d = c.shape[0]
    bits = np.empty(d, np.uint8)
    out = np.empty(7, np.float64)
    lib().orc_quantize_edge(_p(rot), d, _p(c), _p(o), _p(bits), _p(out))
    keys = ("n_o", "alpha", "xc", "f_add", "f_rescale", "f_err", "popcount")
    return bits, dict(zip(keys, out.tolist()))


def estimate_unquantized(rot, c, o, q) -> tuple[float, float, float]:
    """(estimate, bound, exact) in fp64 with an unquantized query."""
    rot, c, o, q = _f32(rot), _f32(c), _f32(o), _f32(q)
    out = np.empty(3, np.float64)
    lib().orc_estimate_unquantized_f64(_p(rot), c.shape[0], _p(c), _p(o), _p(q), _p(out))
    return float(out[0]), float(out[1]), float(out[2])


def exact_dist_f32(q, x) -> float:
    q, x = _f32(q), _f32(x)
    return float(lib().orc_exact_dist_f32(_p(q), _p(x), q.shape[0]))


def sqdist_f64(a, b) -> float:
    a, b = _f32(a), _f32(b)
    return float(lib().orc_sqdist_f64(_p(a), _p(b), a.shape[0]))


def bruteforce(data, q, k: int) -> tuple[np.ndarray, np.ndarray]:
    data, q = _f32(data), _f32(q)
    ids = np.empty(k, np.uint32)
    dd = np.empty(k, np.float64)
    lib().orc_bruteforce(_p(data), data.shape[0], data.shape[1], _p(q), k, _p(ids), _p(dd))
    return ids, dd


def mlp_logit_f32(params, x) -> float:
    params, x = _f32(params), _f32(x)
    return float(lib().orc_mlp_logit_f32(_p(params), _p(x)))


def mlp_loss_grad_f64(params, x, y, w) -> tuple[float, np.ndarray]:
    params = np.ascontiguousarray(params, dtype=np.float64)
    x, y, w = _f32(x), _f32(y), _f32(w)
    g = np.empty(MLP_NPARAM, np.float64)
    loss = lib().orc_mlp_loss_grad_f64(_p(params), _p(x), _p(y), _p(w), x.shape[0], _p(g))
    return float(loss), g


def adam_step_f64(p, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, dtype=np.float64)
    lib().orc_adam_step_f64(_p(p), _p(m), _p(v), _p(g), p.shape[0], t, lr, b1, b2, eps)


def adjust_graph(data, cand, R: int, regular: bool = True) -> tuple[np.ndarray, np.ndarray]:
    """Algorithm 2's "adjust G" (readings R11): each vertex's edge list
    (n x R, sorted by (dist, id), NO_ID after its count) and the counts;
    regular=False: without the angle rule (the "w/o GR" ablation, R17)."""
    data = _f32(data)
    cand = np.ascontiguousarray(cand, dtype=np.uint32)
    n, d = data.shape
    out = np.empty((n, R), np.uint32)
    cnt = np.empty(n, np.uint32)
    rc = lib().orc_adjust_graph(_p(data), n, d, _p(cand), cand.shape[1], R, int(regular), _p(out), _p(cnt))
    if rc != 0:
        raise ValueError(f"oracle adjust_graph failed (code {rc})")
    return out, cnt

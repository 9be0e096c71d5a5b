"""ctypes binding of libsqg.so: the C ABI of include/sqg.h, same names.

Argument marshalling only -- every step of the search runs in the library's
CUDA kernels.  If the shared library is missing the import fails loudly;
there is no CPU fallback.
"""

from __future__ import annotations

import ctypes as C
import pathlib
import threading

PKG = pathlib.Path(__file__).resolve().parent
LIB_PATH = PKG / "_lib" / "libsqg.so"

SQG_OK = 0
SQG_ERR = {-1: "invalid argument", -2: "i/o error", -3: "bad index file format", -4: "out of memory",
           -5: "CUDA error", -6: "bounded device wait expired", -7: "capacity exceeded",
           -8: "unsupported index shape"}
STATUS_CAPACITY, STATUS_LEARNED_STOP, STATUS_BAD_PARAM, STATUS_TIMEOUT = 1, 2, 4, 8
MAX_K, MAX_EF = 256, 2048
MAX_SHARDS = 32
NO_ID = 0xFFFFFFFF
GRAPH_IRREGULAR = 1  # sqg_build_graph_ex: the degree-unaligned "w/o GR" graph
MLP_IN, MLP_HIDDEN, MLP_NPARAM = 16, 64, 5313


class SqgError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {SQG_ERR.get(code, 'unknown error')} ({code})")


class SearchParams(C.Structure):
    _fields_ = [("eps0", C.c_float), ("multi_estimate", C.c_int32), ("hop_cap", C.c_int32),
                ("max_k", C.c_int32), ("max_ef", C.c_int32), ("stop_mlp", C.c_void_p),
                ("stop_logit", C.c_float), ("stop_every", C.c_int32), ("team", C.c_int32),
                ("warps_per_block", C.c_int32), ("timing_events", C.c_void_p * 2),
                ("visited_smem_log2", C.c_int32), ("prefetch", C.c_int32), ("lean", C.c_int32),
                ("rotation", C.c_int32), ("kernel", C.c_int32), ("uniform_k", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("n", C.c_uint64), ("d", C.c_uint32), ("degree", C.c_uint32), ("block_bytes", C.c_uint32),
                ("entry", C.c_uint32), ("off_codes", C.c_uint32), ("off_factors", C.c_uint32),
                ("off_ids", C.c_uint32), ("device", C.c_int32), ("device_bytes", C.c_uint64),
                ("metric", C.c_uint32), ("version", C.c_uint32)]


_lock = threading.Lock()
_lib = None

P, I32, U32, U64, F32, SZ = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_float, C.c_size_t
_SIGS = {
    "sqg_error_string": (C.c_char_p, [I32]),
    "sqg_index_load": (I32, [C.c_char_p, I32, C.POINTER(P)]),
    "sqg_index_free": (None, [P]),
    "sqg_index_info": (I32, [P, C.POINTER(Info)]),
    "sqg_workspace_size": (SZ, [P, I32, I32, I32]),
    "sqg_workspace_size_ex": (SZ, [P, I32, I32, I32, P]),
    "sqg_search": (I32, [P, P, I32, P, P, P, P, P]),
    "sqg_search_ex": (I32, [P, P, I32, P, P, P, P, C.POINTER(SearchParams), P, SZ, P, P]),
    "sqg_search_trace": (I32, [P, P, I32, P, P, P, P, C.POINTER(SearchParams), P, P, I32, P, P, P, I32, P, I32,
                              P]),
    "sqg_prepare_queries": (I32, [P, P, I32, P, P, P, P]),
    "sqg_prepare_queries_tc": (I32, [P, P, I32, P, P, P, P, P]),
    "sqg_estimate_block": (I32, [P, P, I32, P, F32, P, P, P, P, P]),
    "sqg_get_status": (I32, [P, P, C.POINTER(U32)]),
    "sqg_knn_host": (I32, [P, U64, U32, U32, P, I32]),
    "sqg_build_graph": (I32, [P, U64, U32, P, U32, U32, U32, U64, P, P, I32]),
    "sqg_build_graph_ex": (I32, [P, U64, U32, P, U32, U32, U32, U64, U32, P, P, I32, I32]),
    "sqg_wait_selftest": (I32, [I32, P, P]),
    "sqg_medoid": (U32, [P, U64, U32, I32]),
    "sqg_write_index": (I32, [C.c_char_p, P, U64, U32, P, U32, P, U32, U64, U64, I32]),
    "sqg_write_index2": (I32, [C.c_char_p, P, U64, U32, P, U32, P, U32, U64, U64, I32, U32, U32]),
    "sqg_search_noalloc": (I32, [P, P, I32, P, P, I32, I32, P, P, P]),
    "sqg_noalloc_scratch_bytes": (SZ, []),
    "sqg_merge_topk": (I32, [P, P, I32, I32, I32, P, P, P, P]),
    "sqg_mlp_grad": (I32, [P, P, P, P, I32, P, P, P, P]),
    "sqg_mlp_adam": (I32, [P, P, P, P, I32, F32, F32, F32, F32, P]),
    "sqg_mlp_forward": (I32, [P, P, I32, P, P]),
}


def lib() -> C.CDLL:
    """The loaded libsqg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not LIB_PATH.exists():
                raise ImportError(f"libsqg.so not found at {LIB_PATH}: run __graft_entry__.build() or "
                                  "python -m paper_2411_12229_gb300.build (no CPU fallback exists)")
            L = C.CDLL(str(LIB_PATH))
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name, None)
                if f is None:  # reported by the export test; calls fail loudly
                    continue
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def check(rc: int, what: str) -> None:
    if rc != SQG_OK:
        raise SqgError(rc, what)

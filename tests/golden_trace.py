"""Reader of tests/golden/beam_trace_d32.txt, the hand-worked trace of
Algorithm 1 below the full beam, and the index file it describes.

The fixture states the vertices by their coefficients on five Hadamard
axes (x_v = q + sum_i a_v[i] h_i, h_i = row i of the 32 x 32 Sylvester
Hadamard matrix), the tree's edges, and what Algorithm 1 does on it at
ef = 1..4, derived by hand: the beam after each expansion, the expansion
order, the results and the learned-stop features f5 and f6.
"""

from __future__ import annotations

import pathlib
from fractions import Fraction

import numpy as np

PATH = pathlib.Path(__file__).with_name("golden") / "beam_trace_d32.txt"
NO_ID = 0xFFFFFFFF


def hadamard(n: int) -> np.ndarray:
    """Sylvester's construction: H_1 = [1], H_2m = [[H, H], [H, -H]]."""
    h = np.ones((1, 1), dtype=np.int64)
    while h.shape[0] < n:
        h = np.block([[h, h], [h, -h]])
    return h


def load() -> dict:
    t = {"vertex": {}, "edges": [], "beam": {}, "path": {}, "result": {}, "stop": {}}
    for line in PATH.read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "q":
            t["q"] = np.array(f[1:], dtype=np.int64)
        elif f[0] == "vertex":
            t["vertex"][f[1]] = {"id": int(f[2]), "a": np.array(f[3:8], dtype=np.int64), "D": int(f[8])}
        elif f[0] == "edge":
            t["edges"].append((f[1], f[2]))
        elif f[0] == "entry":
            t["entry"] = f[1]
        elif f[0] == "beam":
            ents = []
            for e in f[3:]:
                vis = e.endswith("*")
                e = e.rstrip("*")
                name = e.rstrip("0123456789")
                ents.append((name, int(e[len(name):]), vis))
            t["beam"][(int(f[1]), int(f[2]))] = ents
        elif f[0] == "path":
            t["path"][int(f[1])] = f[2:]
        elif f[0] == "result":
            t["result"][int(f[1])] = f[2:]
        elif f[0] == "stop":
            t["stop"].setdefault(int(f[1]), []).append((int(f[2]), Fraction(f[3]), Fraction(f[4])))
        elif f[0] == "feat":
            t.setdefault("feat", {}).setdefault((int(f[1]), int(f[2])), []).append(
                (int(f[3]), [Fraction(v) for v in f[4:20]]))
    return t


def vectors(t: dict) -> np.ndarray:
    """x_v = q + sum_i a_v[i] h_i, as an (n, 32) integer array by vertex id."""
    h = hadamard(32)[1:6]
    n = len(t["vertex"])
    x = np.zeros((n, 32), dtype=np.int64)
    for v in t["vertex"].values():
        x[v["id"]] = t["q"] + v["a"] @ h
    return x


def adjacency(t: dict, R: int = 32) -> np.ndarray:
    """Both directions of every tree edge; unused slots empty (NO_ID)."""
    n = len(t["vertex"])
    lists = [[] for _ in range(n)]
    for u, v in t["edges"]:
        a, b = t["vertex"][u]["id"], t["vertex"][v]["id"]
        lists[a].append(b)
        lists[b].append(a)
    adj = np.full((n, R), NO_ID, dtype=np.uint32)
    for u, l in enumerate(lists):
        adj[u, :len(l)] = l
    return adj


def write_index(t: dict, path) -> None:
    """The fixture as an index file: identity rotation, entry r."""
    from paper_2411_12229_gb300 import index_builder as ib
    ib.write_index(path, vectors(t).astype(np.float32), adjacency(t), np.eye(32, dtype=np.float32),
                   t["vertex"][t["entry"]]["id"], 0, 0)


def names(t: dict) -> dict:
    """vertex id -> name."""
    return {v["id"]: k for k, v in t["vertex"].items()}

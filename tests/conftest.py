import os
import pathlib
import sys

import numpy as np
import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300); parity tests through the C ABI")
    config.addinivalue_line("markers", "slow: long-running")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if gpu_available():
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def lib_built():
    """The library, built in-tree (host part usable without a GPU)."""
    from paper_2411_12229_gb300 import build
    build.build()
    from paper_2411_12229_gb300 import _binding
    return _binding.lib()


@pytest.fixture(scope="session")
def tiny_index(tmp_path_factory, lib_built, oracle_mod):
    """A 2,000-vertex, d=128, R=32 index from the tiny workload's recipe,
    built on the host from an exact kNN graph; returns (path, data, queries)."""
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300 import synth
    w = synth.small(synth.TINY_10K_D128, 2000, 64)
    x = synth.base(w)
    q = synth.queries(w)
    p = tmp_path_factory.mktemp("idx") / "tiny.sqg"
    ib.build_index(p, x, 32)
    return p, x, q


@pytest.fixture(scope="session")
def tiny_index_r64(tmp_path_factory, lib_built, oracle_mod):
    """A 1,000-vertex, d=64, R=64 index (two neighbours per lane)."""
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300 import synth
    w = synth.small(synth.HIGHDIM_1M_D960.with_(d=64), 1000, 32)
    x = synth.base(w)
    q = synth.queries(w)
    p = tmp_path_factory.mktemp("idx64") / "tiny64.sqg"
    ib.build_index(p, x, 64)
    return p, x, q

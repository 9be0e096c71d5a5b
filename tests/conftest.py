import pathlib
import sys

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


SHAPES = {  # name: (workload, n, d, R): the other workloads' vector shapes at small n
    "highdim-d960-R64": ("highdim-1m-d960", 3000, 960, 64),
    "uneven-d1536-R32": ("uneven-1m-d1536", 2000, 1536, 32),
    "serving-d96-R32": ("serving-4m-d96", 4000, 96, 32),
    "d256-R32": ("batched-1m-d128", 2000, 256, 32),
}


@pytest.fixture(scope="session", params=list(SHAPES))
def shaped_index_file(request, tmp_path_factory, lib_built):
    """Small indexes of the other workloads' shapes, built with the GPU
    search iterations; returns (path, data, queries)."""
    from paper_2411_12229_gb300 import index_builder as ib
    from paper_2411_12229_gb300 import synth
    name, n, d, R = SHAPES[request.param]
    w = synth.small(synth.WORKLOADS[name].with_(d=d), n, 48)
    x, q = synth.base(w), synth.queries(w)
    p = tmp_path_factory.mktemp(request.param) / "s.sqg"
    ib.build_index(p, x, R, device=0, init="random", iterations=2, ef_build=48)
    return p, x, q

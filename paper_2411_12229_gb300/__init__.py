"""GB300-native query phase of SymphonyQG (arXiv 2411.12229).

``api.Index`` loads an index file onto a GPU and searches batches of queries
with the library's CUDA kernels (Algorithm 1 with multiple estimated
distances and implicit re-ranking).  ``index_builder.build_index`` writes
index files (Algorithm 2).  ``synth`` draws the seeded synthetic workloads.
"""

import importlib

from ._binding import (MAX_EF, MAX_K, MLP_NPARAM, NO_ID, STATUS_BAD_PARAM,  # noqa: F401
                       STATUS_CAPACITY, STATUS_LEARNED_STOP, STATUS_TIMEOUT, SqgError)


def __getattr__(name):
    # torch-dependent parts load on first use so host-only tools import fast
    if name == "Index":
        return importlib.import_module(".api", __name__).Index
    raise AttributeError(name)

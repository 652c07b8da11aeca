"""Shared test set-up: import path, the ``gpu`` marker, cached systems."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


# Module order: the hot path first (its oracle pins, then its GPU parity),
# then the rows built on it, so that under -x a failure in a later row never
# hides the hot path's result.  Modules not listed keep their place after
# these, in name order.
_ORDER = ("test_abi", "test_oracle_", "test_gpu_parity", "test_gpu_golden", "test_gpu_batch", "test_gpu_scf",
          "test_gpu_force", "test_gpu_cnn", "test_gpu_warmstart")


def _rank(item):
    name = os.path.basename(str(getattr(item, "path", None) or item.fspath))
    for i, prefix in enumerate(_ORDER):
        if name.startswith(prefix):
            return i
    return len(_ORDER)


def pytest_collection_modifyitems(session, config, items):
    items.sort(key=_rank)             # stable: keeps the order inside a module


@pytest.fixture(scope="session")
def synth_cache():
    import synth
    cache = {}

    def get(name):
        if name not in cache:
            cache[name] = synth.make_system(name)
        return cache[name]
    return get

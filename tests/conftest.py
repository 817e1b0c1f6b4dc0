"""Shared pytest configuration: the ``gpu`` marker and cached seeded workloads."""
import functools
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@functools.lru_cache(maxsize=None)
def cached_workload(name, **kw):
    from paper_2509_04666_gb300 import workloads as W
    return getattr(W, name)(**kw)


@pytest.fixture(scope="session")
def mb1k():
    return cached_workload("mb1k")


@pytest.fixture(scope="session")
def mb1k_dense():
    # test-only variant: half of the frames pointed near bodies (many hits)
    return cached_workload("mb1k", n_bodies=1000, n_frames=400, dense_frac=0.5)

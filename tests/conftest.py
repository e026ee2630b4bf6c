import os
import sys
import functools

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libmpmc.so")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


@functools.lru_cache(maxsize=None)
def links(dims, kind="haar", seed=0, eps=0.3):
    from paper_2306_09559_gb300 import synth
    return synth.gauge_field(dims, kind=kind, seed=seed, eps=eps)


@functools.lru_cache(maxsize=None)
def operator(dims, kind="haar", seed=0, kappa=0.12, eps=0.3, bc_t=1):
    from oracle.lattice import WilsonOperator
    return WilsonOperator(links(dims, kind, seed, eps), kappa, bc_t)


@functools.lru_cache(maxsize=None)
def dense(dims, kind="haar", seed=0, kappa=0.12, eps=0.3, bc_t=1):
    from oracle.lattice import dense_A
    return dense_A(links(dims, kind, seed, eps), kappa, bc_t)


@pytest.fixture
def rng():
    return np.random.Generator(np.random.PCG64(12345))

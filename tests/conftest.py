"""Shared fixtures. GPU tests carry the ``gpu`` marker; everything else runs on the CPU."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")


@pytest.fixture(scope="session")
def ora():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def synth():
    from paper_2302_02733_gb300 import synth as s

    return s


@pytest.fixture(scope="session")
def torus_grid(synth):
    """The full-size seeded torus grid (288 x 128 x 128 x 8 float32) and its description."""
    return synth.fm_torus_grid(1)


@pytest.fixture(scope="session")
def small_grid(synth):
    """A coarse grid (48 x 32 x 16) built the same way, for quick oracle checks."""
    return synth.fm_torus_grid(3, grid=synth.GridParams(n1=48, n2=32, n3=16))

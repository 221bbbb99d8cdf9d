"""Shared test set-up: markers, import paths, the oracle and its references."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a)")


@pytest.fixture(scope="session")
def oracle_lib():
    from oracle import oracle
    return oracle.default()


@pytest.fixture(scope="session")
def philox_ref():
    pytest.importorskip("triton")
    import oracle_pins
    return oracle_pins.reference_tables()

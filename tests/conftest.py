import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def build_library():
    """Compile libmess.so (loads paper_2406_03121_gb300/build.py by path) and return its path."""
    import importlib.util
    path = os.path.join(ROOT, "paper_2406_03121_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("_mess_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


@pytest.fixture(scope="session")
def mess():
    build_library()
    import paper_2406_03121_gb300 as m
    return m

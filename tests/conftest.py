import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def orc():
    """The oracle; SCPL_ORACLE_DIR names another copy of the oracle package
    (the mutation test runs the pins against copies with a planted error)."""
    path = os.environ.get("SCPL_ORACLE_DIR")
    if path:
        import importlib.util
        spec = importlib.util.spec_from_file_location(
            "oracle_under_test", os.path.join(path, "__init__.py"),
            submodule_search_locations=[path])
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()
        return mod
    import oracle
    oracle.build()
    return oracle

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def golden(name: str) -> str:
    with open(os.path.join(GOLDEN, name)) as f:
        return f.read()


@pytest.fixture(scope="session")
def oracle_mod():
    alt = os.environ.get("PBN_ORACLE_DIR")
    if alt:
        # a copy of the oracle with a planted mistake (tests/test_oracle_mutants.py)
        import importlib.util
        spec = importlib.util.spec_from_file_location("oracle_under_test", os.path.join(alt, "oracle.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
    else:
        from oracle import oracle as mod
    mod.build()
    return mod

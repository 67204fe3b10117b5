import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built decoder library")


@pytest.fixture(scope="session", autouse=True)
def _built_cpu_libs():
    import oracle
    from paper_2605_00038_gb300 import _build
    oracle.build()
    _build.build_synth()
    yield

import os
import re
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture
def work_dir(request):
    """A scratch directory inside the repository (tests/_tmp/<test>), emptied
    before the test; tests write no files outside the repository."""
    name = re.sub(r"[^A-Za-z0-9_.-]", "_", request.node.name)[:80]
    d = os.path.join(ROOT, "tests", "_tmp", name)
    shutil.rmtree(d, ignore_errors=True)
    os.makedirs(d)
    return d

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def host_lib(tmp_path_factory):
    """The library's CUDA-free host builders (csrc/pattern.cpp and
    csrc/layouts.cpp) with the test entry points of tests/layout_shim.cpp,
    compiled by g++ into a shared library."""
    import ctypes
    import subprocess
    csrc = os.path.join(ROOT, "paper_1309_5048_gb300", "csrc")
    out = tmp_path_factory.mktemp("hostlib") / "libhost.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-I", csrc,
                    os.path.join(ROOT, "tests", "layout_shim.cpp"), os.path.join(csrc, "layouts.cpp"),
                    os.path.join(csrc, "pattern.cpp"), "-o", str(out)], check=True)
    return ctypes.CDLL(str(out))


def read_golden(name):
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            s = line.strip()
            if not s or s.startswith("#"):
                continue
            rows.append(s.split())
    return rows

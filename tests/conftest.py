import ctypes
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU-only oracle run")


@pytest.fixture(scope="session")
def host_shim(tmp_path_factory):
    """The library's host-only sources (linear algebra, Chebyshev-filter ellipses, grid axes, tensor-core
    operands) with the test-only C wrappers of tests/host_shim.cpp, compiled by g++ into a temporary
    shared object (no CUDA runtime)."""
    out = tmp_path_factory.mktemp("hostshim") / "libhostshim.so"
    csrc = os.path.join(ROOT, "paper_2210_08816_gb300", "csrc")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", f"-I{cuda}/include", f"-I{csrc}",
           os.path.join(ROOT, "tests", "host_shim.cpp"), os.path.join(csrc, "host_linalg.cpp"),
           os.path.join(csrc, "host_cheb.cpp"), os.path.join(csrc, "host_grid.cpp"),
           os.path.join(csrc, "host_tc.cpp"), "-o", str(out)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return ctypes.CDLL(str(out))

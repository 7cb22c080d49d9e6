"""The host-side table validator (csrc/tami_validate.cpp) accepts a real table and refuses each
single-field corruption of it (an index out of range, a slot read before it is written, a leaf
run that overruns its node, a section past the blob).  A C++ harness is compiled against
libtami's internal header and run; it needs no GPU."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2311_17189_gb300")


def test_validator_refuses_corrupted_tables(tmp_path):
    lib = os.path.join(PKG, "libtami.so")
    if not os.path.exists(lib):
        pytest.skip("libtami.so not built")
    exe = str(tmp_path / "validate_cases")
    cmd = ["g++", "-std=c++17", "-O1", os.path.join(ROOT, "tests", "native", "validate_cases.cpp"),
           "-I", os.path.join(PKG, "csrc"), "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include",
           "-L", PKG, "-ltami", "-Wl,-rpath," + PKG, "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("refused") == 17

"""Host logic checked by C++ harnesses against libtami's internal header (no GPU): nothing throws
across the C ABI (the guard around the host-allocating entry points turns an exception into a
status and a message), and the pole DAG's distinct chain prefixes (dag_prefixes) on a hand-built
program."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2311_17189_gb300")


def test_exceptions_become_statuses(tmp_path):
    if not os.path.exists(os.path.join(PKG, "libtami.so")):
        pytest.skip("libtami.so not built")
    exe = str(tmp_path / "guard_cases")
    cmd = ["g++", "-std=c++17", "-O1", os.path.join(ROOT, "tests", "native", "guard_cases.cpp"),
           "-I", os.path.join(PKG, "csrc"), "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include",
           "-L", PKG, "-ltami", "-Wl,-rpath," + PKG, "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    print(r.stdout)
    assert r.returncode == 0 and r.stdout.count("ok ") == 5, r.stdout + r.stderr


def test_dag_prefixes_on_a_hand_built_program(tmp_path):
    if not os.path.exists(os.path.join(PKG, "libtami.so")):
        pytest.skip("libtami.so not built")
    exe = str(tmp_path / "dag_prefix_cases")
    cmd = ["g++", "-std=c++17", "-O1", os.path.join(ROOT, "tests", "native", "dag_prefix_cases.cpp"),
           "-I", os.path.join(PKG, "csrc"), "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include",
           "-L", PKG, "-ltami", "-Wl,-rpath," + PKG, "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    print(r.stdout)
    assert r.returncode == 0 and "0 failures" in r.stdout, r.stdout + r.stderr

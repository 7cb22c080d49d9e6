"""The disk cache of compiled specialised kernels (csrc/tami_jit.cpp): a C++ harness compiled
against libtami's internal header writes an entry, reads it back, and checks that a foreign
identity and every kind of damage to the file are refused before a cubin would reach the driver.
It needs no GPU (the bytes it caches are never loaded)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2311_17189_gb300")


def test_cache_entries_are_verified(tmp_path):
    lib = os.path.join(PKG, "libtami.so")
    if not os.path.exists(lib):
        pytest.skip("libtami.so not built")
    exe = str(tmp_path / "jit_cache_cases")
    cmd = ["g++", "-std=c++17", "-O1", os.path.join(ROOT, "tests", "native", "jit_cache_cases.cpp"),
           "-I", os.path.join(PKG, "csrc"), "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include",
           "-L", PKG, "-ltami", "-Wl,-rpath," + PKG, "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    scratch = tmp_path / "scratch"
    scratch.mkdir()
    r = subprocess.run([exe, str(scratch)], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("refused") == 16 and r.stdout.count("accepted") == 6
    assert "0 failures" in r.stdout

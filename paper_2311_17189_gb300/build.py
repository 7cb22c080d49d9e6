"""Build libtami.so in-tree for sm_103a (GB300).

The host sources (g++) and the kernels (nvcc, -gencode arch=compute_103a,code=sm_103a) are
compiled in parallel, then linked with nvcc into paper_2311_17189_gb300/libtami.so.  The text of
csrc/tami_devmath.cuh is also embedded as a string (_build/tami_devmath_src.inc) for the kernels
that tami_jit.cpp generates and compiles with NVRTC at run time.  No cmake.
"""
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
BUILD = os.path.join(PKG, "_build")
OUT = os.path.join(PKG, "libtami.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SOURCES = ["tami_host.cpp", "tami_graph.cpp", "tami_validate.cpp", "tami_jit.cpp", "tami_cuda.cu", "tami_bwd.cu",
           "tami_batch.cu"]
HEADERS = ["tami_internal.h", "tami_device.cuh", "tami_devmath.cuh", "tami_fwd_tile.cuh"]


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _embed_devmath():
    """Write csrc/tami_devmath.cuh as a C++ raw string literal (kDevmathSource), if it changed."""
    with open(os.path.join(CSRC, "tami_devmath.cuh")) as f:
        text = f.read()
    assert ")TAMIDEV\"" not in text
    inc = ("// generated by build.py from csrc/tami_devmath.cuh\n"
           "static const char kDevmathSource[] = R\"TAMIDEV(" + text + ")TAMIDEV\";\n")
    path = os.path.join(BUILD, "tami_devmath_src.inc")
    if not os.path.exists(path) or open(path).read() != inc:
        with open(path, "w") as f:
            f.write(inc)


def build(force=False, verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    _embed_devmath()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "tami.h")]
    objs, procs = [], []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if not force and not _stale(obj, [path] + hdrs + [__file__]):
            continue
        if src.endswith(".cu"):
            cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", INCLUDE, "-c", path, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
        else:
            cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-I", INCLUDE, "-I", BUILD,
                   "-I", "/usr/local/cuda/include", "-c", path, "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            sys.stderr.write(out.decode())
            raise RuntimeError("compile failed: " + " ".join(cmd))
        if verbose and out:
            sys.stderr.write(out.decode())
    if force or procs or _stale(OUT, objs):
        cmd = [NVCC, *ARCH, "-shared", "-cudart", "static", "-o", OUT + ".tmp", *objs, "-ldl"]
        subprocess.run(cmd, check=True)
        os.replace(OUT + ".tmp", OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

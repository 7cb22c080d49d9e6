"""The specialised fused kernels (tami_jit_source): the generated CUDA C++ compiles with NVRTC for
sm_103a for a spread of tables -- the bench's order-4 table, the order-2 bosonic-transfer table,
a fourth-order pole (Fermi derivatives up to f^(4) in the adjoint), order-5 tables and a table
with a frequency-free group and real denominators -- and diagrams outside the generator's limits
are refused.  NVRTC runs on the host, so no GPU is needed; skipped where libnvrtc is absent."""
import ctypes
import os

import numpy as np
import pytest

import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import _lib as L
from paper_2311_17189_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2311_17189_gb300", "csrc", "tami_devmath.cuh")


def nvrtc():
    for name in ("libnvrtc.so.13", "/usr/local/cuda/lib64/libnvrtc.so.13"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libnvrtc not available")


def compile_cubin(src):
    nv = nvrtc()
    prog = ctypes.c_void_p()
    hdr = open(HEADER).read().encode()
    assert nv.nvrtcCreateProgram(ctypes.byref(prog), src.encode(), b"k.cu", 1, (ctypes.c_char_p * 1)(hdr),
                                 (ctypes.c_char_p * 1)(b"tami_devmath.cuh")) == 0
    opts = [b"-arch=sm_103a", b"-std=c++17", b"-w"]
    rc = nv.nvrtcCompileProgram(prog, len(opts), (ctypes.c_char_p * len(opts))(*opts))
    n = ctypes.c_size_t()
    nv.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    log = ctypes.create_string_buffer(n.value)
    nv.nvrtcGetProgramLog(prog, log)
    m = ctypes.c_size_t()
    nv.nvrtcGetCUBINSize(prog, ctypes.byref(m))
    nv.nvrtcDestroyProgram(ctypes.byref(prog))
    return rc, log.value.decode(), m.value


def tables():
    c = W.ORDER4
    d4 = next(x for x in T.enumerate_sigma(4) if x["code"] == tuple(c["code"]))
    d5 = next(x for x in T.enumerate_sigma(5) if x["code"] == tuple(W.ORDER5["code"]))
    return [
        ("order4_bench", T.Diagram(d4["alpha"], eps=d4["eps"])),
        ("order2_bosonic", T.Diagram(W.ORDER2["alpha"], var_is_boson=W.ORDER2["var_is_boson"])),
        ("quadruple_pole", T.Diagram([[1, 0], [1, 0], [1, 0], [1, 0], [1, 1]],
                                     eps=[[1, 0, 0, 0, 0]] * 4 + [[0, 0, 0, 0, 1]], var_is_boson=[0, 1])),
        ("order5_largest", T.Diagram(d5["alpha"], eps=d5["eps"])),
        ("order3_first", T.Diagram(T.enumerate_sigma(3)[0]["alpha"], eps=T.enumerate_sigma(3)[0]["eps"])),
    ]


KERNEL = {"fused": "tami_jit_fused", "forward": "tami_jit_fwd", "adjoint": "tami_jit_bwd", "energy": "tami_jit_energy"}


@pytest.mark.parametrize("kind", ["fused", "forward", "adjoint", "energy"])
@pytest.mark.parametrize("name,D", tables(), ids=[t[0] for t in tables()])
def test_generated_kernel_compiles_for_sm103a(name, D, kind):
    src = D.jit_source(kind)
    assert KERNEL[kind] in src and "__launch_bounds__" in src
    rc, log, cubin = compile_cubin(src)
    assert rc == 0, log[:3000]
    assert cubin > 0


@pytest.mark.parametrize("env", [{"TAMI_JIT_FIRSTTERM": "0"}, {"TAMI_JIT_PSFIRST": "0"}, {"TAMI_JIT_PSMUL": "fwd"},
                                 {"TAMI_JIT_PSMUL": "all"}, {"TAMI_JIT_PSMUL": "0"}],
                         ids=["firstterm0", "psfirst0", "psmul_fwd", "psmul_all", "psmul0"])
def test_measured_variants_still_compile(env, monkeypatch):
    """The generator's A/B switches (read when a source is generated) give kernels that compile, on
    a small and a large table, so the variants measured against the defaults stay buildable; the
    default source differs from the variant where the switch applies."""
    small, large = tables()[0][1], tables()[3][1]
    base = {n: D.jit_source("fused") for n, D in (("small", small), ("large", large))}
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    changed = False
    for n, D in (("small", small), ("large", large)):
        src = D.jit_source("fused")
        changed |= src != base[n]
        rc, log, cubin = compile_cubin(src)
        assert rc == 0 and cubin > 0, (n, log[:3000])
    assert changed


def test_kinds_differ_only_where_they_should():
    """The forward kernel carries no adjoint sweep, the adjoint no forward sums."""
    D = tables()[0][1]
    fwd, adj, fused = D.jit_source("forward"), D.jit_source("adjoint"), D.jit_source("fused")
    assert "fvbar" not in fwd and "accX" not in fwd and "accV" in fwd
    assert "accV" not in adj and "fvbar" in adj and "saved[" in adj
    assert "fvbar" in fused and "accV" in fused


FREQ_FREE = [[1, 0], [1, 0]]   # sum_nu G1 G2 with no external frequency: R = 1, one real denominator


def test_generator_covers_frequency_free_groups_and_real_denominators():
    """A table whose terms carry no external frequency (R = 1, the frequency-free group first) and
    a frequency-independent denominator E1 - E2: the generator writes those paths and the result
    compiles.  (The enumerated self-energy tables all carry the external frequency.)"""
    D = T.Diagram(FREQ_FREE)
    i = D.info()
    assert i["n_real_dens"] == 1 and i["n_cplx_dens"] == 0
    src = D.jit_source()
    assert "Wb2_0 = s_gsum" in src
    rc, log, _ = compile_cubin(src)
    assert rc == 0, log[:3000]


def test_several_externals_energy_input_only():
    """Momentum sampling takes one external; the energy-input kind takes several (its frequency
    rows are combined per external-coefficient vector) and its source compiles."""
    for alpha, boson, n_ext in (([[1, 1, 0], [1, 0, 1]], None, 2),
                                ([[1, 1, 0, 0], [1, 0, 1, 0], [1, 0, 0, 1]], [0, 1, 0, 0], 3)):
        D = T.Diagram(alpha, var_is_boson=boson, n_ext=n_ext)
        for kind in ("fused", "forward", "adjoint"):
            with pytest.raises(L.TamiError) as e:
                D.jit_source(kind)
            assert e.value.code == L.TAMI_EUNSUPPORTED
        src = D.jit_source("energy")
        assert "kJitXvec" in src
        rc, log, _ = compile_cubin(src)
        assert rc == 0, log[:3000]


def test_jit_mode_argument_checked():
    assert L.lib().tami_set_jit(3) == L.TAMI_EINVAL
    assert L.lib().tami_set_jit(-1) == L.TAMI_EINVAL
    T.set_jit("auto")
    with pytest.raises(L.TamiError):
        L.check(L.lib().tami_jit_source(tables()[0][1]._h, 4, None, 0, None))

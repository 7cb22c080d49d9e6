"""ctypes binding of libtami (include/tami.h): argument marshalling only.

Every numeric step runs in libtami's CUDA kernels or its host construction code.  PyTorch is
used for device memory and for the current CUDA stream.  If libtami.so has not been built the
import fails loudly; there is no fallback path.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtami.so")

TAMI_OK, TAMI_EINVAL, TAMI_ENOMEM, TAMI_ECUDA, TAMI_ETIMEOUT, TAMI_EUNSUPPORTED = range(6)
TAMI_JIT_NEVER, TAMI_JIT_AUTO, TAMI_JIT_ALWAYS = range(3)
TAMI_STAGING_AUTO, TAMI_STAGING_STREAMED = range(2)

# functions declared in include/tami.h (checked by tests/test_lib_host.py)
EXPORTS = [
    "tami_last_error", "tami_construct", "tami_construct_ext", "tami_label_graph", "tami_construct_from_graph", "tami_diagram_info", "tami_upload", "tami_sample_energies",
    "tami_eval_energies", "tami_forward_workspace", "tami_forward", "tami_forward_noalloc",
    "tami_backward_workspace", "tami_backward", "tami_forward_backward_workspace", "tami_forward_backward",
    "tami_set_jit", "tami_jit_prepare", "tami_jit_status", "tami_jit_source", "tami_jit_cached",
    "tami_batch_plan", "tami_batch_info", "tami_batch_launch",
    "tami_batch_destroy", "tami_batch_debug_set_item", "tami_batch_specialised",
    "tami_enumerate_sigma",
    "tami_set_table_staging", "tami_debug_set_wait_limit",
    "tami_selftest_exp", "tami_selftest_sincos", "tami_selftest_imul", "tami_selftest_imul_ftz", "tami_selftest_fp64_rate", "tami_destroy",
]


class TamiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libtami error {code}: {msg}")
        self.code = code


class Lattice(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("tp", ctypes.c_double), ("mu", ctypes.c_double),
                ("kx_ext", ctypes.c_double), ("ky_ext", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [
        ("n_lines", ctypes.c_int), ("n_vars", ctypes.c_int),
        ("n_terms", ctypes.c_int64), ("n_fermi_factors", ctypes.c_int64), ("n_g_factors", ctypes.c_int64),
        ("max_der", ctypes.c_int), ("max_g", ctypes.c_int),
        ("unique_poles", ctypes.c_int64), ("unique_dens", ctypes.c_int64),
        ("n_combos", ctypes.c_int), ("n_fermi_values", ctypes.c_int), ("n_real_dens", ctypes.c_int),
        ("n_cplx_dens", ctypes.c_int), ("n_groups_fixed", ctypes.c_int), ("n_groups_freq", ctypes.c_int),
        ("table_bytes", ctypes.c_int),
        ("flops_per_sample", ctypes.c_double), ("flops_per_sample_freq", ctypes.c_double),
        ("bwd_flops_per_sample", ctypes.c_double), ("bwd_flops_per_sample_freq", ctypes.c_double),
        ("saved_rows", ctypes.c_int),
        ("fwd_save_flops_per_sample", ctypes.c_double), ("bwd_saved_flops_per_sample", ctypes.c_double),
        ("fused_flops_per_sample_freq", ctypes.c_double),
        ("n_ext", ctypes.c_int),
        ("energy_in_flops_per_sample", ctypes.c_double),
        ("energy_in_flops_per_sample_freq", ctypes.c_double),
        ("n_dag_ops", ctypes.c_int), ("n_dag_nodes", ctypes.c_int), ("n_phase2_factors", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, u64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
    L.tami_last_error.restype = ctypes.c_char_p
    L.tami_construct.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, ctypes.c_double, ctypes.POINTER(vp)]
    L.tami_construct_ext.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, ctypes.c_double,
                                     ctypes.POINTER(vp)]
    L.tami_label_graph.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.tami_construct_from_graph.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(vp)]
    L.tami_diagram_info.argtypes = [vp, ctypes.POINTER(Info)]
    L.tami_upload.argtypes = [vp, ctypes.c_int, vp]
    L.tami_sample_energies.argtypes = [vp, ctypes.POINTER(Lattice), u64, u64, i64, dp, vp]
    L.tami_eval_energies.argtypes = [vp, dp, i64, dp, ctypes.c_int, ctypes.c_double, dp, vp]
    L.tami_forward_workspace.argtypes = [vp, i64, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    L.tami_forward.argtypes = [vp, ctypes.POINTER(Lattice), u64, u64, i64, dp, ctypes.c_int, ctypes.c_double,
                               dp, dp, dp, dp, dp, ctypes.c_size_t, vp]
    L.tami_forward_noalloc.argtypes = [vp, ctypes.POINTER(Lattice), u64, u64, i64, dp, ctypes.c_int,
                                       ctypes.c_double, dp, dp, dp, vp]
    L.tami_backward_workspace.argtypes = [vp, i64, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    L.tami_backward.argtypes = [vp, ctypes.POINTER(Lattice), u64, u64, i64, dp, ctypes.c_int, ctypes.c_double,
                                dp, dp, dp, dp, dp, dp, dp, dp, ctypes.c_size_t, vp]
    L.tami_forward_backward_workspace.argtypes = [vp, i64, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    L.tami_forward_backward.argtypes = [vp, ctypes.POINTER(Lattice), u64, u64, i64, dp, ctypes.c_int, ctypes.c_double,
                                        dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, ctypes.c_size_t, vp]
    L.tami_set_jit.argtypes = [ctypes.c_int]
    L.tami_jit_prepare.argtypes = [vp]
    L.tami_jit_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_double)]
    L.tami_jit_source.argtypes = [vp, ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.tami_jit_cached.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.tami_batch_plan.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
    L.tami_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int)]
    L.tami_batch_launch.argtypes = [vp, ctypes.POINTER(Lattice), dp, ctypes.c_double, dp, dp, vp]
    L.tami_batch_specialised.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.tami_batch_destroy.argtypes = [vp]
    L.tami_batch_debug_set_item.argtypes = [vp, ctypes.c_int, ctypes.c_int, i64, i64, ctypes.POINTER(ctypes.c_int64)]
    L.tami_batch_debug_set_item.restype = ctypes.c_int
    L.tami_batch_destroy.restype = None
    L.tami_enumerate_sigma.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int)]
    L.tami_set_table_staging.argtypes = [ctypes.c_int, ctypes.c_int]
    L.tami_debug_set_wait_limit.argtypes = [i64]
    L.tami_selftest_exp.argtypes = [dp, i64, dp, dp, dp, vp]
    L.tami_selftest_sincos.argtypes = [dp, i64, dp, dp, vp]
    L.tami_selftest_imul.argtypes = [dp, dp, i64, dp, vp]
    L.tami_selftest_imul_ftz.argtypes = [dp, dp, i64, dp, vp]
    L.tami_selftest_fp64_rate.argtypes = [ctypes.c_int, ctypes.c_int, i64, dp, ctypes.POINTER(ctypes.c_double), vp]
    L.tami_destroy.argtypes = [vp]
    L.tami_destroy.restype = None
    _lib = L
    return L


def check(rc):
    if rc != TAMI_OK:
        raise TamiError(rc, lib().tami_last_error().decode())


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)

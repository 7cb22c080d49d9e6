"""tami_forward_noalloc: the forward evaluation for callers that cannot allocate device memory
(its scratch is a fixed array inside libtami).  Called through the C ABI and compared with
tami_forward, which uses a caller-allocated workspace, on two calls in a row; plus the size
limit and a smaller call after a larger one (the shared array keeps the previous contents).

This file is collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import _lib as L
from paper_2311_17189_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-11


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    c = W.ORDER4
    d = next(x for x in T.enumerate_sigma(4) if x["code"] == tuple(c["code"]))
    D = T.Diagram(d["alpha"], eps=d["eps"]).upload(0)
    return c, D


def call_noalloc(D, c, n, X, offset=0):
    dev = "cuda:0"
    Xd = torch.view_as_real(torch.as_tensor(X, dtype=torch.complex128, device=dev)).contiguous()
    n_f = Xd.shape[0]
    mean = torch.full((n_f, 2), float("nan"), dtype=torch.float64, device=dev)
    var = torch.full((n_f, 2), float("nan"), dtype=torch.float64, device=dev)
    lat = L.Lattice(*[float(v) for v in W.lattice(c)])
    rc = L.lib().tami_forward_noalloc(D._h, ctypes.byref(lat), c["seed"], offset, n,
                                      ctypes.c_void_p(Xd.data_ptr()), n_f, c["beta"],
                                      ctypes.c_void_p(mean.data_ptr()), ctypes.c_void_p(var.data_ptr()), None,
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, mean.cpu().numpy(), var.cpu().numpy()


def reference(D, c, n, X, offset=0):
    mean, var, ps = D.forward(W.lattice(c), c["seed"], offset, n, X, c["beta"], per_sample=True)
    torch.cuda.synchronize()
    ps = torch.view_as_real(ps).cpu().numpy()
    return torch.view_as_real(mean).cpu().numpy(), var.cpu().numpy(), np.abs(ps).mean(axis=1)


def test_noalloc_matches_workspace_entry_twice(setup):
    c, D = setup
    X = W.matsubara(c["beta"], c["n_freq"])
    n = 1 << 20
    ref_mean, ref_var, scale = reference(D, c, n, X)
    for _ in range(2):
        rc, mean, var = call_noalloc(D, c, n, X)
        assert rc == L.TAMI_OK, L.lib().tami_last_error().decode()
        assert np.all(np.abs(mean - ref_mean) <= RTOL * scale)
        assert np.allclose(var, ref_var, rtol=1e-10, atol=0)


def test_noalloc_smaller_call_after_larger_one(setup):
    c, D = setup
    X = W.matsubara(c["beta"], 4)
    for n in (200_000, 1000):
        ref_mean, ref_var, scale = reference(D, c, n, X, offset=7)
        rc, mean, var = call_noalloc(D, c, n, X, offset=7)
        assert rc == L.TAMI_OK, L.lib().tami_last_error().decode()
        assert np.all(np.abs(mean - ref_mean) <= RTOL * scale)
        assert np.allclose(var, ref_var, rtol=1e-10, atol=0)


def test_noalloc_rejects_sizes_beyond_its_array(setup):
    """A request whose scratch (the same size tami_forward would need, tami_forward_workspace) is
    above the fixed 4 MiB array is refused with TAMI_EINVAL and nothing launched."""
    c, D = setup
    X = W.real_axis(-4.0, 4.0, 2048, 0.05)
    n = 1 << 20
    need = ctypes.c_size_t()
    L.check(L.lib().tami_forward_workspace(D._h, n, len(X), ctypes.byref(need)))
    assert need.value > 4 << 20
    rc, _, _ = call_noalloc(D, c, n, X)
    assert rc == L.TAMI_EINVAL
    assert "scratch" in L.lib().tami_last_error().decode()

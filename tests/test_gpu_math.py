"""The kernels' own elementary functions against CUDA's: the table-driven exponential for t <= 0
(e^t and e^t - 1, after Tang, ACM TOMS 1989) against torch.exp / torch.expm1 on the device
(CUDA's exp/expm1), and against mpmath at a few points."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2311_17189_gb300 import _lib as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def selftest(t):
    t = t.to(device="cuda", dtype=torch.float64).contiguous()
    y = torch.empty_like(t)
    em = torch.empty_like(t)
    yp = torch.empty_like(t)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.check(L.lib().tami_selftest_exp(ctypes.c_void_p(t.data_ptr()), t.numel(), ctypes.c_void_p(y.data_ptr()),
                                      ctypes.c_void_p(em.data_ptr()), ctypes.c_void_p(yp.data_ptr()), s))
    torch.cuda.synchronize()
    # the variant without e^t - 1 (used for the Fermi-type segments) gives the same bits
    assert torch.equal(yp.view(torch.int64), y.view(torch.int64))
    return y, em


def test_exp_neg_against_cuda_exp_and_expm1():
    rng = np.random.default_rng(0)
    t = np.concatenate([
        -np.logspace(-300, np.log10(1400.0), 400001),          # tiny to deep tail
        -rng.uniform(0, 1, 200000), -rng.uniform(0, 50, 200000),
        -np.arange(0, 2000) * np.log(2) / 32,                 # table boundaries
        [0.0, -0.0, -1e-320, -708.0, -709.9, -745.0, -746.0, -1400.0],
    ])
    tt = torch.tensor(t, dtype=torch.float64)
    y, em = selftest(tt)
    ry, rem = torch.exp(tt.cuda()), torch.expm1(tt.cuda())
    normal = ry > 1e-289
    rel_y = ((y - ry).abs() / ry)[normal]
    assert rel_y.max().item() <= 3.4e-16
    deep = (ry <= 1e-289) & (ry > 1e-300)
    assert (((y - ry).abs() / ry)[deep]).max().item() <= 2e-15
    assert torch.all(y[ry == 0] <= 5e-324)          # at most one denormal ulp at the underflow edge
    rel_em = ((em - rem).abs() / rem.abs())[rem != 0]
    assert rel_em.max().item() <= 3.4e-16
    assert torch.all(em[tt.cuda() == 0] == 0) and torch.all(y[tt.cuda() == 0] == 1)


def test_exp_neg_against_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    t = np.array([-1e-12, -3e-5, -0.0108, -0.0217, -0.5, -1.0, -7.25, -33.3, -200.0, -700.0])
    y, em = selftest(torch.tensor(t))
    y, em = y.cpu().numpy(), em.cpu().numpy()
    for i, ti in enumerate(t):
        ey = mp.exp(mp.mpf(float(ti)))
        assert abs(y[i] - float(ey)) <= 3e-16 * float(ey)
        assert abs(em[i] - float(ey - 1)) <= 3e-16 * abs(float(ey - 1))

"""The kernels' own elementary functions: the table-driven exponential for t <= 0 (e^t and
e^t - 1, after Tang, ACM TOMS 1989) against torch.exp / torch.expm1 on the device (CUDA's
exp/expm1) and against mpmath at a few points; the Cody-Waite cos/sin of the dispersion against
the C library's (the oracle's), which fixes TRIG_ERR of the momentum-mode parity bounds; the
integer-pipe product against the FP64 unit's; and the FP64 fma-rate probe's flop count against its
own outputs."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2311_17189_gb300 import _lib as L

import bounds as B

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
        -np.arange(0, 16000) * np.log(2) / 256,               # table boundaries
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


def test_sincos_against_c_library():
    """Kernel cos/sin within TRIG_ERR (3e-16, absolute) of the C library's, which the oracle's
    dispersion uses (itself pinned to one ulp of 50-digit values), over the range of line momenta
    a lattice sample produces (|k| up to about 7 pi) and beyond; exact at 0; the cosine-only path
    of the energies gives the sin/cos path's bits.  The bound is absolute: one polynomial on
    [-pi/2, pi/2], whose Horner sum 1 + z p(z) cancels near the zeros of cos (the dispersion
    needs only absolute accuracy)."""
    rng = np.random.default_rng(3)
    k = np.concatenate([np.linspace(-7 * np.pi, 7 * np.pi, 400001), rng.uniform(-22.0, 22.0, 200000),
                        np.array([0.0, -0.0, np.pi / 2, -np.pi / 2, np.pi, 1e-300, -1e-8])])
    kt = torch.tensor(k, device="cuda")
    st = torch.empty_like(kt)
    ct = torch.empty_like(kt)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.check(L.lib().tami_selftest_sincos(ctypes.c_void_p(kt.data_ptr()), kt.numel(), ctypes.c_void_p(st.data_ptr()),
                                         ctypes.c_void_p(ct.data_ptr()), s))
    torch.cuda.synchronize()
    sg, cg = st.cpu().numpy(), ct.cpu().numpy()
    assert np.all(np.isfinite(cg)), "cosine-only path differs from the sin/cos path"
    so, co = O.sincos(k)
    es, ec = np.max(np.abs(sg - so)), np.max(np.abs(cg - co))
    print(f"kernel sin/cos against the C library: max abs diff {es:.2e} / {ec:.2e}")
    assert es <= B.TRIG_ERR and ec <= B.TRIG_ERR
    assert sg[-7] == 0.0 and cg[-7] == 1.0


# (recurrences per thread, steps per trip, own multiplier and addend per recurrence, running sum)
RATE_VARIANTS = [(8, 8, False, False), (4, 8, True, False), (4, 16, True, True), (3, 16, True, False)]


@pytest.mark.parametrize("variant", range(len(RATE_VARIANTS)))
def test_fp64_rate_probe_does_its_work(variant):
    """Every operand pattern of the FP64 rate probe: the recurrences a_k <- m_k a_k + c_k (or the
    running sums a_k <- m_k c_k + a_k) from known starts give each thread the closed-form sum to
    rounding, so the timed launch does all the flops it reports; a variant out of range is refused."""
    blocks, trips = 4, 1000
    C, U, own, acc = RATE_VARIANTS[variant]
    out = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    fl = ctypes.c_double()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.check(L.lib().tami_selftest_fp64_rate(variant, blocks, trips, ctypes.c_void_p(out.data_ptr()), ctypes.byref(fl), s))
    torch.cuda.synchronize()
    assert fl.value == 2.0 * C * U * trips * 256 * blocks
    m, c, steps = 0.9999999, 1e-3, U * trips
    t = np.arange(blocks * 256)
    ref = np.zeros(blocks * 256)
    for k in range(C):
        mk, ck = (m - 1e-9 * k, c + 1e-9 * k) if own else (m, c)
        a0 = 1e-3 * ((t + k) & 1023)
        ref += a0 + steps * (mk * ck) if acc else a0 * mk ** steps + ck * (1 - mk ** steps) / (1 - mk)
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-9, atol=0)
    assert L.lib().tami_selftest_fp64_rate(len(RATE_VARIANTS), blocks, trips, ctypes.c_void_p(out.data_ptr()),
                                           ctypes.byref(fl), s) == L.TAMI_EINVAL


def special_operands(rng, n):
    """Pairs of doubles across the whole range: random normals over all exponents, close exponents,
    near-cancelling pairs, rounding ties, results that underflow or overflow, zeros of both signs,
    subnormals, infinities and NaNs."""
    def rnd(k, lo, hi):
        m = rng.uniform(1.0, 2.0, k) * np.where(rng.random(k) < 0.5, -1.0, 1.0)
        return np.ldexp(m, rng.integers(lo, hi, k))
    a = [rnd(n, -1022, 1023)]
    b = [rnd(n, -1022, 1023)]
    x = rnd(n, -60, 60)                                             # close exponents
    a.append(x); b.append(x * np.ldexp(1.0, rng.integers(-70, 70, n)) * rng.uniform(0.5, 2.0, n))
    a.append(x); b.append(-x * (1.0 + np.ldexp(rng.integers(-8, 8, n).astype(float), -52)))   # cancellation
    a.append(x); b.append(-x)                                       # exact zero sums
    a.append(np.ldexp(1.0 + np.ldexp(rng.integers(0, 2**20, n).astype(float), -52), 0))
    b.append(np.ldexp(1.0 - np.ldexp(rng.integers(0, 2**20, n).astype(float), -53), 0))   # rounding ties
    tiny = rnd(n, -1074, -1000)
    huge = rnd(n, 1000, 1023)
    a.append(tiny); b.append(rnd(n, -60, 0))                        # underflowing products
    a.append(huge); b.append(rnd(n, 0, 60))                         # overflowing products
    sp = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, np.inf, -np.inf, np.nan, 1.0, -1.0,
                   1.7976931348623157e308, np.ldexp(1.0, -1022), np.ldexp(1.5, -1023)])
    aa, bb = np.meshgrid(sp, np.concatenate([sp, rnd(20, -1022, 1023)]))
    a.append(aa.ravel()); b.append(bb.ravel())
    return np.concatenate(a), np.concatenate(b)


def test_integer_pipe_product_is_ieee():
    """The kernels' integer-pipe product (imul) equals the FP64 unit's DMUL bit for bit (NaNs as
    NaNs) on operands across the whole double range and its special cases."""
    rng = np.random.default_rng(11)
    a, b = special_operands(rng, 400000)
    at, bt = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
    mul = torch.empty_like(at)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.check(L.lib().tami_selftest_imul(ctypes.c_void_p(at.data_ptr()), ctypes.c_void_p(bt.data_ptr()), at.numel(),
                                       ctypes.c_void_p(mul.data_ptr()), s))
    torch.cuda.synchronize()
    for got, ref, what in ((mul, at * bt, "product"),):
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        nan = np.isnan(r)
        assert np.array_equal(np.isnan(g), nan), what
        bad = g[~nan].view(np.uint64) != r[~nan].view(np.uint64)
        assert not bad.any(), (what, a[~nan][bad][:5], b[~nan][bad][:5], g[~nan][bad][:5], r[~nan][bad][:5])


def test_integer_pipe_product_ftz():
    """The call-free integer-pipe product (imul_ftz) on the same operands: the IEEE product (from
    numpy) bit for bit wherever both operands are normal and the product is normal; a signed zero
    for a zero or subnormal operand or a product below 2^-1022 (at exactly 2^-1022, where the
    unrounded product may lie just below, either); a signed infinity for an overflowing product
    or an infinite operand against a normal one; a NaN for a NaN operand or infinity times a zero
    or subnormal."""
    rng = np.random.default_rng(12)
    a, b = special_operands(rng, 400000)
    at, bt = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
    mul = torch.empty_like(at)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.check(L.lib().tami_selftest_imul_ftz(ctypes.c_void_p(at.data_ptr()), ctypes.c_void_p(bt.data_ptr()),
                                           at.numel(), ctypes.c_void_p(mul.data_ptr()), s))
    torch.cuda.synchronize()
    g = mul.cpu().numpy()
    tiny = np.ldexp(1.0, -1022)
    with np.errstate(all="ignore"):
        r = a * b
    sign = np.signbit(a) ^ np.signbit(b)
    fin_a, fin_b = np.isfinite(a), np.isfinite(b)
    sub_a, sub_b = fin_a & (np.abs(a) < tiny), fin_b & (np.abs(b) < tiny)
    nan_ref = np.isnan(a) | np.isnan(b) | (np.isinf(a) & sub_b) | (np.isinf(b) & sub_a)
    assert np.array_equal(np.isnan(g), nan_ref)
    ok = ~nan_ref
    inf_in = (np.isinf(a) | np.isinf(b)) & ok
    assert np.all(np.isinf(g[inf_in])) and np.array_equal(np.signbit(g[inf_in]), sign[inf_in])
    fin = ok & ~inf_in
    flush = fin & (sub_a | sub_b | (np.abs(r) < tiny))
    assert np.all(g[flush] == 0.0) and np.array_equal(np.signbit(g[flush]), sign[flush])
    edge = fin & ~flush & (np.abs(r) == tiny)
    assert np.all((g[edge] == 0.0) | (g[edge] == r[edge]))
    rest = fin & ~flush & ~edge
    bad = g[rest].view(np.uint64) != r[rest].view(np.uint64)
    assert not bad.any(), (a[rest][bad][:5], b[rest][bad][:5], g[rest][bad][:5], r[rest][bad][:5])

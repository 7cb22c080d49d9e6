"""GPU parity of the adjoint (tami_backward) against the oracle's forward-mode dual numbers and
against central finite differences of the GPU forward mean.

Per-sample bound: 1e-11 times the oracle's derivative rounding envelope (the product rule
applied to the magnitudes of every factor and its derivative), the analogue of the value
envelope used for the forward, plus the input part that allows for the two sides' cos/sin
(tests/bounds.py: the energy sensitivity of the derivative and, for k_ext, of the value).
Contracted gradients sum over frequencies with |g_f|.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import workloads as W

import bounds as B

pytestmark = pytest.mark.gpu

RTOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def both(alpha, eps=None, boson=None, prefactor=1.0):
    D = T.Diagram(alpha, eps=eps, var_is_boson=boson, prefactor=prefactor).upload(0)
    S = O.Solution(alpha, eps=eps, var_is_boson=boson, prefactor=prefactor)
    return D, S


def upstream(n_f, seed=3):
    r = np.random.default_rng(seed)
    return r.normal(size=n_f) + 1j * r.normal(size=n_f)


CASES = [
    # name, order/diagram or explicit alpha, lattice, beta, X
    ("order3_real_axis", 3, 0, (1.0, 0.0, 0.0, np.pi / 2, np.pi / 2), 10.0, W.real_axis(-4.0, 4.0, 7, 0.05)),
    ("order4_matsubara", 4, 2, (1.0, -0.3, -0.5, np.pi / 2, np.pi / 2), 8.0, W.matsubara(8.0, 5)),
    ("order5_real_axis", 5, 7, (1.0, -0.2, 0.1, np.pi / 2, np.pi / 3), 5.0, W.real_axis(-2.0, 2.0, 3, 0.1)),
    # four lines with one momentum label: a fourth-order pole, so the forward needs f^(3) and the
    # adjoint f^(4); the external variable bosonic
    ("quadruple_pole", dict(alpha=[[1, 0], [1, 0], [1, 0], [1, 0], [1, 1]],
                            eps=[[1, 0, 0, 0, 0]] * 4 + [[0, 0, 0, 0, 1]], boson=[0, 1]), None,
     (1.0, -0.3, 0.2, np.pi / 3, np.pi / 5), 2.0, W.real_axis(-3.0, 3.0, 5, 0.1)),
]


def setup_case(case):
    name, order, idx, lat, beta, X = case
    if isinstance(order, dict):
        D, S = both(np.array(order["alpha"]), np.array(order["eps"]), boson=order["boson"])
        assert S.info()["max_der"] == 3
        return D, S, lat, beta, X
    d = O.enumerate_sigma(order)[idx]
    D, S = both(d["alpha"], d["eps"], prefactor=(-1.0) ** order * (-1.0) ** d["loops"])
    return D, S, lat, beta, X


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_per_sample_derivatives_against_dual_numbers(case):
    D, S, lat, beta, X = setup_case(case)
    n, seed, off = 3 * 128 + 37, 21, 5
    g = upstream(len(X))
    out = D.backward(lat, seed, off, n, X, beta, g, per_sample=True)
    torch.cuda.synchronize()
    dX = out["dX"].cpu().numpy()
    grads = out["grads"].cpu().numpy()
    ref, env = B.oracle_deriv(S, lat, seed, off, n, X, beta, "omega")
    assert np.all(np.abs(dX - ref) <= env), np.max(np.abs(dX - ref) / env)
    for k, which in enumerate(("mu", "kx", "ky")):
        der, dbd = B.oracle_deriv(S, lat, seed, off, n, X, beta, which)
        contracted = np.real(np.conj(g)[:, None] * der).sum(axis=0)
        bound = (np.abs(g)[:, None] * dbd).sum(axis=0)
        assert np.all(np.abs(grads[:, k] - contracted) <= bound), (which, np.max(np.abs(grads[:, k] - contracted) / bound))
    # means: dSigma/dX and the contracted gradients
    mdX = out["dSigma_dX"].cpu().numpy()
    assert np.all(np.abs(mdX - ref.mean(axis=1)) <= env.mean(axis=1))
    gX = out["grad_X_re"].cpu().numpy()
    assert np.allclose(gX, np.real(np.conj(g) * mdX), rtol=1e-14, atol=1e-300)
    gp = out["grad_params"].cpu().numpy()
    assert np.all(np.abs(gp - grads.mean(axis=0)) <= 1e-13 * np.abs(grads).mean(axis=0))


def test_adjoint_against_central_differences():
    """grad of L = Re sum_f conj(g_f) Sigma_f by central differences (h = 1e-5) of the GPU
    forward mean on the same samples; truncation error ~h^2, rounding ~1e-16/h."""
    D, S, lat, beta, X = setup_case(CASES[0])
    n, seed = 1 << 16, 4
    g = upstream(len(X))
    out = D.backward(lat, seed, 0, n, X, beta, g)
    gp = out["grad_params"].cpu().numpy()
    gX = out["grad_X_re"].cpu().numpy()
    h = 1e-5

    def L(lt, XX):
        m, _, _ = D.forward(lt, seed, 0, n, XX, beta)
        return np.real(np.conj(g) * m.cpu().numpy())

    for k, idx in enumerate((2, 3, 4)):
        lp, lm = list(lat), list(lat)
        lp[idx] += h
        lm[idx] -= h
        fd = (L(lp, X).sum() - L(lm, X).sum()) / (2 * h)
        assert abs(gp[k] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gX).max()), (k, gp[k], fd)
    fdX = (L(lat, X + h) - L(lat, X - h)) / (2 * h)
    assert np.allclose(gX, fdX, rtol=1e-6, atol=1e-6 * np.abs(gX).max())


def test_autograd_function_matches_direct_calls():
    """SigmaMC (torch.autograd.Function over tami_forward / tami_backward): loss = sum |Sigma|^2;
    autograd's gradients equal tami_backward with g = 2 Sigma, and the value equals forward."""
    from paper_2311_17189_gb300.autograd import SigmaMC
    D, S, lat, beta, X = setup_case(CASES[0])
    n, seed = 1 << 14, 9
    omega = torch.tensor(np.real(X), dtype=torch.float64, device="cuda", requires_grad=True)
    gamma = torch.tensor(0.05, dtype=torch.float64, device="cuda")
    mu = torch.tensor(lat[2], dtype=torch.float64, device="cuda", requires_grad=True)
    kext = torch.tensor(lat[3:5], dtype=torch.float64, device="cuda", requires_grad=True)
    sigma = SigmaMC.apply(D, omega, gamma, mu, kext, lat[0], lat[1], beta, n, seed, 0)
    loss = (sigma.abs() ** 2).sum()
    loss.backward()
    m, _, _ = D.forward(lat, seed, 0, n, X, beta)
    assert torch.allclose(sigma.detach(), m, rtol=0, atol=0)
    ref = D.backward(lat, seed, 0, n, X, beta, 2 * m)
    assert torch.allclose(omega.grad, ref["grad_X_re"], rtol=1e-13, atol=0)
    assert torch.allclose(mu.grad, ref["grad_params"][0], rtol=1e-13, atol=0)
    assert torch.allclose(kext.grad, ref["grad_params"][1:3], rtol=1e-13, atol=0)


def test_order3_real_axis_full_size_sampled():
    """Order-3 self-energy on the real axis at its full size (2^22 samples, 256 frequencies
    omega + 0.05i on [-4, 4], beta = 10): per-sample contracted gradients at 300 random samples
    against the oracle computed one by one, and the means against the mean of the per-sample
    outputs."""
    c = W.ORDER3_REAL
    d = O.enumerate_sigma(c["order"])[c["diagram_index"]]
    D, S = both(d["alpha"], d["eps"])
    X = W.real_axis(*c["omega"], c["gamma"])
    g = upstream(len(X), seed=5)
    n = c["n_samples"]
    lat = W.lattice(c)
    out = D.backward(lat, c["seed"], 0, n, X, c["beta"], g, per_sample=False)
    torch.cuda.synchronize()
    # per-sample grads at sampled indices: run the per-sample path on single-sample slices
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(n, 300, replace=False))
    for i in idx[:300]:
        o1 = D.backward(lat, c["seed"], int(i), 1, X, c["beta"], g, per_sample=True)
        got = o1["grads"].cpu().numpy()[0]
        for k, which in enumerate(("mu", "kx", "ky")):
            der, dbd = B.oracle_deriv(S, lat, c["seed"], int(i), 1, X, c["beta"], which, threads=1)
            ref = np.real(np.conj(g) * der[:, 0]).sum()
            assert abs(got[k] - ref) <= (np.abs(g) * dbd[:, 0]).sum()
    # full-size means vs a second, per-sample run of the same launch
    full = D.backward(lat, c["seed"], 0, n, X, c["beta"], g, per_sample=False)
    assert torch.equal(full["grad_params"], out["grad_params"])          # deterministic
    assert torch.equal(full["dSigma_dX"], out["dSigma_dX"])


@pytest.mark.parametrize("beta", W.ORDER5["betas"])
def test_order5_large_full_size_sampled(beta):
    """The large-order workload at its full size: the order-5 diagram with the largest flat table
    (744 terms), 2^26 samples, one frequency i pi/beta.  Forward: per-sample values at 200 random
    samples against the oracle computed one by one, and the mean against the mean of all
    per-sample outputs.  Adjoint (term products recomputed, nothing stored per sample): the
    per-sample dSigma/dX and contracted gradients at 40 random samples against the oracle's dual
    numbers, and a second full launch equal bit for bit."""
    c = W.ORDER5
    d = next(x for x in O.enumerate_sigma(c["order"]) if x["code"] == c["code"])
    D, S = both(d["alpha"], d["eps"])
    assert S.info()["terms"] == D.info()["n_terms"] == 744
    X = W.matsubara(beta, c["n_freq"])
    n = c["n_samples"]
    lat = W.lattice(c)
    mean, var, ps = D.forward(lat, c["seed"], 0, n, X, beta, per_sample=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(int(beta))
    idx = np.sort(rng.choice(n, 200, replace=False))
    got = ps[:, torch.as_tensor(idx, device="cuda")].cpu().numpy()
    plain = []
    for k, i in enumerate(idx):
        r = S.eval_momenta(lat, c["seed"], int(i), 1, X, beta, per_sample=True)
        err = np.abs(got[:, k] - r["values"][:, 0])
        assert np.all(err <= B.value_bound(r, lat)[:, 0]), (i, err, r["envelope"][:, 0])
        plain.append(np.mean(err <= RTOL * np.abs(r["values"][:, 0])))
    print(f"order-5 workload, beta {beta}: {np.mean(plain):.4f} of sampled values within plain relative 1e-11")
    ps_mean = ps.mean(dim=1).cpu().numpy()
    scale = ps.abs().mean(dim=1).cpu().numpy()
    assert np.all(np.abs(mean.cpu().numpy() - ps_mean) <= 1e-12 * scale)
    del ps
    g = np.array([1.0 + 0.5j])
    out = D.backward(lat, c["seed"], 0, n, X, beta, g, per_sample=False)
    again = D.backward(lat, c["seed"], 0, n, X, beta, g, per_sample=False)
    assert torch.equal(out["grad_params"], again["grad_params"])
    assert torch.equal(out["dSigma_dX"], again["dSigma_dX"])
    assert np.all(np.isfinite(out["grad_params"].cpu().numpy()))
    for i in idx[:40]:
        o1 = D.backward(lat, c["seed"], int(i), 1, X, beta, g, per_sample=True)
        gs = o1["grads"].cpu().numpy()[0]
        dref, dbd = B.oracle_deriv(S, lat, c["seed"], int(i), 1, X, beta, "omega", threads=1)
        assert np.all(np.abs(o1["dX"].cpu().numpy()[:, 0] - dref[:, 0]) <= dbd[:, 0])
        for k, which in enumerate(("mu", "kx", "ky")):
            der, dbd = B.oracle_deriv(S, lat, c["seed"], int(i), 1, X, beta, which, threads=1)
            ref = np.real(np.conj(g) * der[:, 0]).sum()
            assert abs(gs[k] - ref) <= (np.abs(g) * dbd[:, 0]).sum(), (i, which, gs[k], ref)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_saved_energies_give_the_same_bits(case):
    """tami_forward with `saved` (line energies and dE/dK factors per sample) and tami_backward
    reading them give exactly the results of the recomputing path: the forward's outputs, the
    per-sample adjoints and the reduced gradients, bit for bit."""
    D, S, lat, beta, X = setup_case(case)
    n, seed, off = 3 * 128 + 37, 21, 5
    g = upstream(len(X))
    sv = D.saved_buffer(n)
    m0, v0, p0 = D.forward(lat, seed, off, n, X, beta, per_sample=True)
    m1, v1, p1 = D.forward(lat, seed, off, n, X, beta, per_sample=True, save=sv)
    assert torch.equal(m0, m1) and torch.equal(v0, v1) and torch.equal(p0, p1)
    # the leading rows are line energies: each equals one line's tami_sample_energies column bit for bit
    Eb = D.sample_energies(lat, seed, off, n).cpu().numpy().T.copy().view(np.uint64)
    n_energy_rows = len({col.tobytes() for col in Eb})
    for row in sv.cpu().numpy()[:n_energy_rows].copy().view(np.uint64):
        assert any(np.array_equal(row, col) for col in Eb)
    b0 = D.backward(lat, seed, off, n, X, beta, g, per_sample=True)
    b1 = D.backward(lat, seed, off, n, X, beta, g, per_sample=True, saved=sv)
    for k in ("dSigma_dX", "grad_X_re", "grad_params", "dX", "grads"):
        assert torch.equal(b0[k], b1[k]), k


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fused_forward_backward(case):
    """tami_forward_backward (forward and adjoint in one pass): each sample's value, dv/dX and
    contracted gradients equal the separate tami_forward / tami_backward outputs bit for bit; the
    reduced mean, variance, dSigma/dX and gradients agree with them to the rounding of the sums
    (the two launches group the partial sums differently)."""
    D, S, lat, beta, X = setup_case(case)
    n, seed, off = 3 * 128 + 37, 21, 5
    g = upstream(len(X))
    m, v, p = D.forward(lat, seed, off, n, X, beta, per_sample=True)
    b = D.backward(lat, seed, off, n, X, beta, g, per_sample=True)
    fb = D.forward_backward(lat, seed, off, n, X, beta, g, per_sample=True)
    torch.cuda.synchronize()
    assert torch.equal(fb["values"], p)
    assert torch.equal(fb["dX"], b["dX"]) and torch.equal(fb["grads"], b["grads"])
    scale = p.abs().mean(dim=1)
    assert torch.all((fb["mean"] - m).abs() <= 1e-13 * scale)
    assert torch.allclose(fb["var"], v, rtol=1e-12, atol=0)
    dscale = b["dX"].abs().mean(dim=1)
    assert torch.all((fb["dSigma_dX"] - b["dSigma_dX"]).abs() <= 1e-13 * dscale)
    gscale = b["grads"].abs().mean(dim=0)
    assert torch.all((fb["grad_params"] - b["grad_params"]).abs() <= 1e-13 * gscale)


def test_order4_fused_full_size_sampled():
    """The benchmark's launch at its full size: the fused forward + adjoint over 2^24 samples of
    the order-4 workload with the bench's upstream gradient.  Per-sample values and contracted
    gradients at 300 random samples against the oracle computed one by one; the means against
    the means of the per-sample outputs."""
    c = W.ORDER4
    d = next(x for x in O.enumerate_sigma(4) if x["code"] == c["code"])
    D, S = both(d["alpha"], d["eps"])
    X, lat, beta, n = W.matsubara(c["beta"], c["n_freq"]), W.lattice(c), c["beta"], c["n_samples"]
    g = np.ones(len(X)) + 0.5j
    out = D.forward_backward(lat, c["seed"], 0, n, X, beta, g, per_sample=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(4)
    idx = np.sort(rng.choice(n, 300, replace=False))
    ti = torch.as_tensor(idx, device="cuda")
    vals = out["values"][:, ti].cpu().numpy()
    grads = out["grads"][ti].cpu().numpy()
    for k, i in enumerate(idx):
        r = S.eval_momenta(lat, c["seed"], int(i), 1, X, beta, per_sample=True)
        assert np.all(np.abs(vals[:, k] - r["values"][:, 0]) <= B.value_bound(r, lat)[:, 0]), i
        for j, which in enumerate(("mu", "kx", "ky")):
            der, dbd = B.oracle_deriv(S, lat, c["seed"], int(i), 1, X, beta, which, threads=1)
            ref = np.real(np.conj(g) * der[:, 0]).sum()
            assert abs(grads[k, j] - ref) <= (np.abs(g) * dbd[:, 0]).sum(), (i, which)
    scale = out["values"].abs().mean(dim=1)
    assert torch.all((out["mean"] - out["values"].mean(dim=1)).abs() <= 1e-12 * scale)
    gscale = out["grads"].abs().mean(dim=0)
    assert torch.all((out["grad_params"] - out["grads"].mean(dim=0)).abs() <= 1e-12 * gscale)
    dscale = out["dX"].abs().mean(dim=1)
    assert torch.all((out["dSigma_dX"] - out["dX"].mean(dim=1)).abs() <= 1e-12 * dscale)

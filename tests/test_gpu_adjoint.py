"""GPU parity of the adjoint (tami_backward) against the oracle's forward-mode dual numbers and
against central finite differences of the GPU forward mean.

Per-sample bound: 1e-11 times the oracle's derivative rounding envelope (the product rule
applied to the magnitudes of every factor and its derivative), the analogue of the value
envelope used for the forward.  Contracted gradients sum over frequencies with |g_f|.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import workloads as W

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
]


def setup_case(case):
    name, order, idx, lat, beta, X = case
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
    _, ref, env = S.eval_momenta_deriv(lat, seed, off, n, X, beta, "omega", threads=8, envelope=True)
    assert np.all(np.abs(dX - ref) <= RTOL * env), np.max(np.abs(dX - ref) / env)
    for k, which in enumerate(("mu", "kx", "ky")):
        _, der, denv = S.eval_momenta_deriv(lat, seed, off, n, X, beta, which, threads=8, envelope=True)
        contracted = np.real(np.conj(g)[:, None] * der).sum(axis=0)
        bound = RTOL * (np.abs(g)[:, None] * denv).sum(axis=0)
        assert np.all(np.abs(grads[:, k] - contracted) <= bound), (which, np.max(np.abs(grads[:, k] - contracted) / bound))
    # means: dSigma/dX and the contracted gradients
    mdX = out["dSigma_dX"].cpu().numpy()
    assert np.all(np.abs(mdX - ref.mean(axis=1)) <= RTOL * env.mean(axis=1))
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
            _, der, denv = S.eval_momenta_deriv(lat, c["seed"], int(i), 1, X, c["beta"], which, envelope=True)
            ref = np.real(np.conj(g) * der[:, 0]).sum()
            assert abs(got[k] - ref) <= RTOL * (np.abs(g) * denv[:, 0]).sum()
    # full-size means vs a second, per-sample run of the same launch
    full = D.backward(lat, c["seed"], 0, n, X, c["beta"], g, per_sample=False)
    assert torch.equal(full["grad_params"], out["grad_params"])          # deterministic
    assert torch.equal(full["dSigma_dX"], out["dSigma_dX"])

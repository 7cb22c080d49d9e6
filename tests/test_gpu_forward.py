"""GPU parity of the forward path (CUDA kernels through the C ABI) against the CPU oracle.

Tolerances.  With energy input both sides read the same energies; they differ only in the
rounding of exp/expm1, the reciprocals and the order of products and sums.  Each of those is a
relative error of a few ulp on a factor, so the per-sample error is bounded by a small multiple
of 2^-53 times the rounding envelope sum_t |A_t| prod env(FT factors) prod |G| that the oracle
returns; the tests allow 1e-11 of it (the relative 1e-11 of the target, scaled to the terms that
cancel).  In momentum mode the two sides' energies also differ by their cos/sin (the oracle uses
the C library's, the kernels their own), by at most dE; the bound adds twice dE times the
oracle's energy sensitivity (tests/bounds.py).  Monte Carlo means are compared to 1e-11 of
(mean bound / 1e-11 + mean |value|): the first bounds the mean of the per-sample errors, the
second the summation (sample-to-sample cancellation makes |mean| itself the wrong scale).
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


def lib_and_oracle(alpha, eps=None, boson=None, prefactor=1.0, order=None):
    D = T.Diagram(alpha, eps=eps, var_is_boson=boson, prefactor=prefactor, order=order).upload(0)
    S = O.Solution(alpha, eps=eps, var_is_boson=boson, prefactor=prefactor, order=order)
    return D, S


def diagram(order, index=None, code=None):
    ds = O.enumerate_sigma(order)
    if code is not None:
        return next(d for d in ds if d["code"] == tuple(code))
    return ds[index]


def check_per_sample(gpu, ref, env, what, pert=0.0):
    """|gpu - ref| <= RTOL env + pert per sample (pert: the input part of the bound in momentum
    mode); returns the share of samples that also meet a plain relative RTOL."""
    gpu = np.asarray(gpu)
    err = np.abs(gpu - ref)
    bound = RTOL * env + pert
    bad = err > bound
    assert not bad.any(), f"{what}: {bad.sum()} of {bad.size} samples off; worst err/env " \
                          f"{np.max(err / np.maximum(env, 1e-300)):.3e}"
    return float(np.mean(err <= RTOL * np.abs(ref)))


# ---------------------------------------------------------------------------- sampling
@pytest.mark.parametrize("order,offset", [(2, 0), (4, 0), (4, (1 << 33) + 12345), (5, 77)])
def test_sampled_energies_within_trig_bound(order, offset):
    """Philox momenta, line momenta and dispersion: every energy within dE of the oracle's (the
    two sides' cos/sin and rounding, tests/bounds.py).  A wrong counter, key, label or sign moves
    energies by O(1), far outside dE."""
    d = diagram(order, 0)
    D = T.Diagram(d["alpha"], eps=d["eps"]).upload(0)
    lat = (1.0, -0.3, -0.5, np.pi / 2, np.pi / 2)
    n = 5000
    Eg = D.sample_energies(lat, W.SEED, offset, n).cpu().numpy()
    Eo, _ = O.sample_energies(d["alpha"], lat, W.SEED, offset, n)
    err = np.abs(Eg - Eo)
    assert np.max(err) <= B.energy_error(lat), (np.max(err), B.energy_error(lat))
    print(f"order {order}: max |E_gpu - E_oracle| = {np.max(err):.2e} (bound {B.energy_error(lat):.2e}), "
          f"{np.mean(err == 0):.3f} equal")


# ---------------------------------------------------------------------------- energy input
ENERGY_CASES = [
    ("paper_order2", [[1, 0, 0], [0, 1, 0], [-1, 1, 1]], None, None, 1.0),
    ("bosonic_q_order2", [[1, 0, 1], [0, 1, 0], [1, 1, 0]], None, [1, 0, 0], 5.0),
    ("quadruple_pole", [[1, 0], [1, 0], [1, 0], [1, 0], [1, 1]], [[1, 0, 0, 0, 0]] * 4 + [[0, 0, 0, 0, 1]],
     [0, 1], 1.2),
]


@pytest.mark.parametrize("case", ENERGY_CASES, ids=[c[0] for c in ENERGY_CASES])
def test_eval_energies_small_cases(case):
    """Energy-input evaluation (Sec. 2.3) on the paper's example workload: energies U(-8, 8),
    fermionic/bosonic frequencies, several tiles and a ragged tail (n_e = 3*128 + 37)."""
    name, alpha, eps, boson, beta = case
    D, S = lib_and_oracle(alpha, eps, boson)
    N = len(alpha)
    E = W.random_energies(3 * 128 + 37, N, a=8.0, seed=11)
    X = W.matsubara(beta, 5) if boson is None or not boson[-1] else 2j * np.pi / beta * np.arange(1, 6)
    ref, _, env = S.eval_energies(E, X, beta)
    gpu = D.eval_energies(torch.tensor(E, device="cuda"), X, beta).cpu().numpy()
    check_per_sample(gpu, ref, env, name)


@pytest.mark.parametrize("order", [3, 4, 5])
def test_eval_energies_enumerated_diagrams(order):
    """Every enumerated diagram of orders 3-5 on random energies (equal-label lines share
    energies), Matsubara and real-axis frequencies."""
    ds = O.enumerate_sigma(order)
    step = max(1, len(ds) // 8)
    for d in ds[::step]:
        D, S = lib_and_oracle(d["alpha"], d["eps"])
        N = d["alpha"].shape[0]
        E = W.random_energies(300, N, a=4.0, seed=order)
        rep = d["eps"].argmax(1)
        E = E[:, rep]
        for X, beta in ((W.matsubara(3.0, 4), 3.0), (W.real_axis(-2.0, 2.0, 3, 0.05), 10.0)):
            ref, _, env = S.eval_energies(E, X, beta)
            gpu = D.eval_energies(torch.tensor(E, device="cuda"), X, beta).cpu().numpy()
            check_per_sample(gpu, ref, env, f"order {order} code {d['code']}")


def test_energy_input_paper_example_full_size():
    """The paper's evaluation example at its own size (Sec. 5.1): 10^6 energy rows U(-8, 8), 100
    fermionic frequencies, beta = 1, the full [n_f][n_e] output (at this size the diagram's
    specialised kernel).  Rows at 2000 random indices against the oracle; a launch over a slice of
    the rows equals that slice of the full output bit for bit on either kernel (each row is
    evaluated by itself), and the generic kernel agrees with it to rounding."""
    c = W.ENERGY_X1
    D, S = lib_and_oracle(c["alpha"])
    E = W.random_energies(c["n_e"], c["alpha"].shape[0], a=c["a"], seed=c["seed"])
    X = W.matsubara(c["beta"], c["n_freq"])
    Ed = torch.tensor(E, device="cuda")
    out = D.eval_energies(Ed, X, c["beta"])
    torch.cuda.synchronize()
    assert tuple(out.shape) == (c["n_freq"], c["n_e"])
    assert D.jit_status()["last_used"]
    rng = np.random.default_rng(2)
    idx = np.sort(rng.choice(c["n_e"], 2000, replace=False))
    got = out[:, torch.as_tensor(idx, device="cuda")].cpu().numpy()
    ref, _, env = S.eval_energies(E[idx], X, c["beta"])
    check_per_sample(got, ref, env, "energy-input example")
    lo, hi = 123_457, 123_457 + 5 * 128 + 3
    try:
        T.set_jit("always")
        part = D.eval_energies(Ed[lo:hi].contiguous(), X, c["beta"])
        assert torch.equal(part, out[:, lo:hi])
        T.set_jit("never")
        gen = D.eval_energies(Ed, X, c["beta"])
        part = D.eval_energies(Ed[lo:hi].contiguous(), X, c["beta"])
        assert torch.equal(part, gen[:, lo:hi])
        ref, _, env = S.eval_energies(E[idx], X, c["beta"])
        assert np.all(np.abs(gen[:, torch.as_tensor(idx, device="cuda")].cpu().numpy() - got) <= RTOL * env)
    finally:
        T.set_jit("auto")


# ---------------------------------------------------------------------------- momentum mode
def run_both(D, S, lat, seed, offset, n, X, beta, threads=8):
    mean, var, ps = D.forward(lat, seed, offset, n, X, beta, per_sample=True)
    torch.cuda.synchronize()
    ref = S.eval_momenta(lat, seed, offset, n, X, beta, per_sample=True, threads=threads)
    return mean.cpu().numpy(), var.cpu().numpy(), ps.cpu().numpy(), ref


def check_mean(mean, var, ps_ref, ref, lat):
    # the mean of per-sample errors is bounded by the mean of the per-sample bounds; the
    # summation itself adds rounding relative to mean |value|
    scale = B.mean_scale(ref, lat)
    assert np.all(np.abs(mean - ref["mean"]) <= RTOL * scale)
    # var = sum (x - mean)^2 / (n-1): per-sample errors dx <= RTOL env move it by at most
    # 2/(n-1) sum |x - mean| dx, plus the rounding of the sums
    n = ps_ref.shape[1]
    dev = ps_ref - ref["mean"][:, None]
    for part, k in ((np.real, 0), (np.imag, 1)):
        tol = 2.0 / max(n - 1, 1) * np.sum(np.abs(part(dev)) * B.value_bound(ref, lat), axis=1) \
            + 1e-10 * ref["var"][:, k]
        assert np.all(np.abs(var[:, k] - ref["var"][:, k]) <= tol)


def test_order2_hubbard_full_workload():
    """Order-2 Hubbard self-energy, full workload: 1e5 samples, beta=5, one frequency; every
    sample and the mean."""
    c = W.ORDER2
    D, S = lib_and_oracle(c["alpha"], boson=c["var_is_boson"])
    X = W.matsubara(c["beta"], c["n_freq"])
    lat = W.lattice(c)
    mean, var, ps, ref = run_both(D, S, lat, c["seed"], 0, c["n_samples"], X, c["beta"])
    frac = check_per_sample(ps, ref["values"], ref["envelope"], "order 2", B.value_pert(ref, lat))
    # share of samples that also meet a plain relative 1e-11; the rest sit where the flat
    # term-by-term form cancels (e.g. f(-E1) - f(-E3) with both close to 1), for both sides
    print(f"order-2 full workload: {frac:.4f} of samples within plain relative 1e-11")
    assert frac > 0.9
    check_mean(mean, var, ref["values"], ref, lat)


@pytest.mark.parametrize("n", [1, 127, 128, 129, 3 * 128 + 37, 4096 + 5])
def test_order4_small_sample_counts(n):
    """Order-4 workload (t'=-0.3, mu=-0.5, beta=8, 16 frequencies) at sample counts around the
    tile size, including a single sample and ragged tails."""
    c = W.ORDER4
    d = diagram(4, code=c["code"])
    D, S = lib_and_oracle(d["alpha"], d["eps"])
    X = W.matsubara(c["beta"], c["n_freq"])
    lat = W.lattice(c)
    mean, var, ps, ref = run_both(D, S, lat, c["seed"], 3, n, X, c["beta"])
    check_per_sample(ps, ref["values"], ref["envelope"], f"order 4 n={n}", B.value_pert(ref, lat))
    check_mean(mean, var, ref["values"], ref, lat)


@pytest.mark.parametrize("n_f", [1, 3, 100, 127, 129, 300])
def test_frequency_counts(n_f):
    """Frequency counts below, at and above the block size: the per-thread frequency split, the
    balanced split of counts that do not divide the block (3, 100, 127) and several frequencies
    per thread (129, 300)."""
    d = diagram(3, 1)
    D, S = lib_and_oracle(d["alpha"], d["eps"])
    X = W.real_axis(-4, 4, n_f, 0.05) if n_f > 3 else W.matsubara(10.0, n_f)
    lat = (1.0, 0.0, 0.0, np.pi / 2, np.pi / 2)
    mean, var, ps, ref = run_both(D, S, lat, 5, 0, 700, X, 10.0)
    check_per_sample(ps, ref["values"], ref["envelope"], f"n_f={n_f}", B.value_pert(ref, lat))
    check_mean(mean, var, ref["values"], ref, lat)


@pytest.mark.parametrize("order", [3, 5])
def test_all_diagrams_momentum_mode(order):
    """Every enumerated diagram of orders 3 and 5 (a sample of them at order 5) with the
    -U^m (-1)^F prefactor, momentum sampling, 2 frequencies."""
    ds = O.enumerate_sigma(order)
    for d in ds[:: max(1, len(ds) // 10)]:
        pref = (-1.0) ** order * (-1.0) ** d["loops"]
        D, S = lib_and_oracle(d["alpha"], d["eps"], prefactor=pref)
        X = W.matsubara(5.0, 2)
        lat = (1.0, -0.2, 0.1, np.pi / 2, np.pi / 3)
        mean, var, ps, ref = run_both(D, S, lat, 9, 1000, 400, X, 5.0)
        check_per_sample(ps, ref["values"], ref["envelope"], f"order {order} {d['code']}", B.value_pert(ref, lat))
        check_mean(mean, var, ref["values"], ref, lat)


def test_order4_full_size_sampled():
    """Order-4 workload at its full size (2^24 samples, 16 frequencies), the launch the
    benchmark times: per-sample values at 2000 random indices against the oracle computed one
    by one, and the mean against the mean of all per-sample outputs."""
    c = W.ORDER4
    d = diagram(4, code=c["code"])
    D, S = lib_and_oracle(d["alpha"], d["eps"])
    X = W.matsubara(c["beta"], c["n_freq"])
    n = c["n_samples"]
    mean, var, ps = D.forward(W.lattice(c), c["seed"], 0, n, X, c["beta"], per_sample=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(n, 2000, replace=False))
    got = ps[:, torch.as_tensor(idx, device="cuda")].cpu().numpy()
    fr = []
    for k, i in enumerate(idx):
        r = S.eval_momenta(W.lattice(c), c["seed"], int(i), 1, X, c["beta"], per_sample=True)
        fr.append(check_per_sample(got[:, k:k + 1], r["values"], r["envelope"], f"sample {i}",
                                   B.value_pert(r, W.lattice(c))))
    print(f"order-4 bench workload: {np.mean(fr):.4f} of sampled values within plain relative 1e-11")
    ps_mean = ps.mean(dim=1).cpu().numpy()
    scale = ps.abs().mean(dim=1).cpu().numpy()
    assert np.all(np.abs(mean.cpu().numpy() - ps_mean) <= 1e-12 * scale)

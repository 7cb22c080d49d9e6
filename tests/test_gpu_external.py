"""GPU parity with several external frequencies (Sec. 2.3: a frequency row holds the diagram's
n_nu external frequencies, the last labels), through energy input, against the CPU oracle; and
the refusal of the momentum-sampling calls for such diagrams (the momentum integrand of Sec. 5.2
appends one external momentum).

Tolerance as in test_gpu_forward.py: per sample 1e-11 of the oracle's rounding envelope
sum_t |A_t| prod env(FT factors) prod |G|.  The kernels form each denominator's external part
as g * (sum_q v_q X_q) once per frequency row, the oracle as sum_q a_q X_q inside every
denominator: a difference of one rounding on a term of the envelope.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import _lib as L
from paper_2311_17189_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def check_per_sample(gpu, ref, env, what):
    err = np.abs(np.asarray(gpu) - ref)
    bad = err > RTOL * env
    assert not bad.any(), f"{what}: {bad.sum()} of {bad.size} values off; worst err/env " \
                          f"{np.max(err / np.maximum(env, 1e-300)):.3e}"


def rows(boson_ext, beta, n_rows=6, real_first=False):
    """Frequency rows [n_rows, n_ext]: Matsubara values of each external's statistics (bosonic
    2 pi i n / beta with n >= 1, fermionic (2n+1) pi i / beta), different per column; with
    real_first the first external is omega + 0.05i on [-2, 2] instead (analytic continuation)."""
    n_ext = len(boson_ext)
    X = np.empty((n_rows, n_ext), dtype=np.complex128)
    for q, b in enumerate(boson_ext):
        n = np.arange(n_rows) * (q + 1) - 2 * q + (1 if b else 0)
        X[:, q] = 1j * (2 * n + (0 if b else 1)) * np.pi / beta
    if real_first:
        X[:, 0] = np.linspace(-2.0, 2.0, n_rows) + 0.05j
    return X


def held(order, k):
    d = O.enumerate_sigma(order)[k]
    return W.hold_external(d["alpha"], order - 1), d["eps"]


CASES = [
    # (name, alpha, eps, var_is_boson, n_ext)
    ("two_fermionic_m1", [[1, 1, 0], [1, 0, 1]], None, None, 2),
    ("one_combination_m1", [[1, 0, 0], [1, 1, -1]], None, None, 2),
    ("three_externals_m1", [[1, 1, 0, 0], [1, 0, 1, 0], [1, 0, 0, 1]], None, [0, 1, 0, 0], 3),
    ("double_pole_m2", [[1, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [-1, 1, 1, 1]],
     [[1, 0, 0, 0], [1, 0, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1]], [0, 0, 1, 0], 2),
    ("sigma3_held", *held(3, 0), None, 2),
    ("sigma4_held", *held(4, 5), None, 2),
]


@pytest.mark.parametrize("real_first", [False, True], ids=["matsubara", "real_axis"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_eval_energies_several_externals(case, real_first):
    """Energy input with n_ext = 2, 3: every (row, frequency row) value against the oracle on
    energies U(-4, 4), several tiles and a ragged tail (n_e = 3*128 + 37); Matsubara rows and rows
    whose first external is continued to omega + i Gamma (nonzero Re X, the general phase 2)."""
    name, alpha, eps, boson, n_ext = case
    alpha = np.asarray(alpha)
    D = T.Diagram(alpha, eps=eps, var_is_boson=boson, n_ext=n_ext).upload(0)
    S = O.Solution(alpha, eps=eps, var_is_boson=boson, n_ext=n_ext)
    beta = 2.0
    bext = [0] * n_ext if boson is None else list(boson[-n_ext:])
    X = rows(bext, beta, real_first=real_first)
    E = W.random_energies(3 * 128 + 37, alpha.shape[0], a=4.0, seed=17)
    ref, _, env = S.eval_energies(E, X, beta)
    gpu = D.eval_energies(torch.tensor(E, device="cuda"), X, beta).cpu().numpy()
    assert gpu.shape == ref.shape
    check_per_sample(gpu, ref, env, name)


def test_one_combination_equals_single_external_on_gpu():
    """An integrand whose two fermionic externals enter only as Omega = nu1 - nu2 (bosonic) gives
    the single-external bubble's values at Omega, through two different tables on the GPU."""
    D2 = T.Diagram([[1, 0, 0], [1, 1, -1]], n_ext=2).upload(0)
    D1 = T.Diagram([[1, 0], [1, 1]], var_is_boson=[0, 1]).upload(0)
    beta = 3.0
    X = rows([0, 0], beta)
    X = X[X[:, 0] != X[:, 1]]
    E = torch.tensor(W.random_energies(1000, 2, a=3.0, seed=5), device="cuda")
    v2 = D2.eval_energies(E, X, beta).cpu().numpy()
    v1 = D1.eval_energies(E, X[:, 0] - X[:, 1], beta).cpu().numpy()
    assert np.allclose(v2, v1, rtol=1e-12, atol=1e-14)


def test_two_external_workload_full_size():
    """The two-external workload at its full size: the order-4 bench diagram with its last loop
    frequency held external, 10^6 energy rows U(-8, 8), the 10 x 10 grid of fermionic (nu', nu),
    beta = 1, the full [100][10^6] output.  Rows at 2000 random indices against the oracle; a
    launch over a slice of the rows equals that slice of the full output bit for bit."""
    c = W.TWO_FREQ_X1
    d = next(x for x in O.enumerate_sigma(c["order"]) if x["code"] == tuple(c["code"]))
    alpha = W.hold_external(d["alpha"], c["held"])
    D = T.Diagram(alpha, eps=d["eps"], n_ext=2).upload(0)
    S = O.Solution(alpha, eps=d["eps"], n_ext=2)
    E = W.random_energies(c["n_e"], alpha.shape[0], a=c["a"], seed=c["seed"])
    X = W.matsubara_grid(c["beta"], c["n_grid"], c["n_grid"])
    Ed = torch.tensor(E, device="cuda")
    out = D.eval_energies(Ed, X, c["beta"])
    torch.cuda.synchronize()
    assert tuple(out.shape) == (c["n_grid"] ** 2, c["n_e"])
    idx = np.sort(np.random.default_rng(3).choice(c["n_e"], 2000, replace=False))
    got = out[:, torch.as_tensor(idx, device="cuda")].cpu().numpy()
    ref, _, env = S.eval_energies(E[idx], X, c["beta"])
    check_per_sample(got, ref, env, "two-external workload")
    lo, hi = 654_321, 654_321 + 3 * 128 + 5
    try:
        T.set_jit("always" if D.jit_status()["last_used"] else "never")   # the kernel the full launch ran
        part = D.eval_energies(Ed[lo:hi].contiguous(), X, c["beta"]).cpu().numpy()
    finally:
        T.set_jit("auto")
    full = out[:, lo:hi].cpu().numpy()
    assert np.array_equal(part.view(np.uint64), full.view(np.uint64))
    del out
    torch.cuda.empty_cache()


def test_momentum_calls_refuse_several_externals():
    """Momentum sampling, the forward and adjoint Monte Carlo calls and batches need n_ext = 1;
    each refuses a two-external diagram with TAMI_EUNSUPPORTED, launches nothing, and the library
    stays usable (a one-external diagram evaluates afterwards)."""
    D = T.Diagram([[1, 1, 0], [1, 0, 1]], n_ext=2).upload(0)
    lat = (1.0, 0.0, 0.0, 0.5, 0.5)
    X = np.array([1j * np.pi])
    calls = [
        lambda: D.sample_energies(lat, 1, 0, 10),
        lambda: D.forward(lat, 1, 0, 256, X, 1.0),
        lambda: D.backward(lat, 1, 0, 256, X, 1.0, np.ones(1, dtype=np.complex128)),
        lambda: D.forward_backward(lat, 1, 0, 256, X, 1.0, np.ones(1, dtype=np.complex128)),
        lambda: T.Batch([D], [256], [1], 1),
    ]
    for call in calls:
        with pytest.raises(L.TamiError) as e:
            call()
        assert e.value.code == L.TAMI_EUNSUPPORTED
        assert "n_ext = 1" in str(e.value)
    c = W.ORDER2
    D1 = T.Diagram(c["alpha"], var_is_boson=c["var_is_boson"]).upload(0)
    mean, _, _ = D1.forward(W.lattice(c), c["seed"], 0, 1000, W.matsubara(c["beta"], 1), c["beta"])
    assert np.all(np.isfinite(mean.cpu().numpy()))

"""Pins of the oracle with several external frequencies (Sec. 2.3: frequency_t rows hold
m + n_nu entries, the n_nu external ones last; each row is one evaluation point).

The expected values come from the plain definition (truncated Matsubara sums over the internal
variables with tail extrapolation, the external frequencies held fixed), from a closed form
derived by partial fractions, and from the reduction of an integrand whose externals enter only
through one combination to the single-external integrand at that combination.
"""
import numpy as np
import pytest

import oracle as O


def n_bose(beta, x):
    return 1.0 / (np.exp(beta * x) - 1.0)


def fermi(beta, x):
    return 1.0 / (np.exp(beta * x) + 1.0)


def extrapolated_sum(alpha, E, X, beta, n_ext, eps=None, boson=None, Ns=(62, 125, 250, 500, 1000, 2000)):
    """Truncated sums on the box |n_l| <= N over the internal variables, extrapolated to
    N -> infinity by fitting the boundary error a/N + (b log N + c)/N^2 + (d log N + e)/N^3."""
    Ns = np.asarray(Ns, dtype=float)
    vals = np.array([O.brute_force(alpha, E, X, beta, int(N), eps=eps, var_is_boson=boson, n_ext=n_ext)
                     for N in Ns])
    M = np.stack([np.ones_like(Ns), 1 / Ns, np.log(Ns) / Ns**2, 1 / Ns**2, np.log(Ns) / Ns**3, 1 / Ns**3], 1)
    return np.linalg.solve(M, vals)[0]


def mats(n, beta, boson=False):
    return 1j * (2 * n + (0 if boson else 1)) * np.pi / beta


def test_two_fermionic_externals_closed_form():
    """(1/beta) sum_nu 1/((i nu + i nu1 + E1)(i nu + i nu2 + E2)), all three frequencies
    fermionic.  Partial fractions give [f(-a) - f(-b)]/(b - a) with a = i nu1 + E1, b = i nu2 + E2,
    and f(x - i nu1) = -n_B(x) for fermionic nu1, so
    I = [n_B(-E2) - n_B(-E1)] / (i nu2 - i nu1 + E2 - E1)."""
    S = O.Solution([[1, 1, 0], [1, 0, 1]], n_ext=2)
    assert S.info()["terms"] == 2
    beta = 2.5
    rng = np.random.default_rng(5)
    E = rng.uniform(0.2, 3.0, (12, 2)) * rng.choice([-1.0, 1.0], (12, 2))
    X = np.array([[mats(0, beta), mats(1, beta)], [mats(-2, beta), mats(3, beta)], [mats(4, beta), mats(-1, beta)]])
    v, _, _ = S.eval_energies(E, X, beta)
    for i in range(E.shape[0]):
        E1, E2 = E[i]
        for fi, (x1, x2) in enumerate(X):
            cf = (n_bose(beta, -E2) - n_bose(beta, -E1)) / (x2 - x1 + E2 - E1)
            assert abs(v[fi, i] - cf) <= 1e-13 * abs(cf)


def test_externals_through_one_combination_reduce_to_one_external():
    """Lines nu and nu + nu1 - nu2 with fermionic nu1, nu2: the integrand depends on the externals
    only through Omega = nu1 - nu2, a bosonic frequency, so its values equal those of the
    single-external bubble (lines nu, nu + Omega, Omega bosonic) at Omega = nu1 - nu2.  The two
    constructions reach it differently (the shift parity sums over two fermionic externals)."""
    S2 = O.Solution([[1, 0, 0], [1, 1, -1]], n_ext=2)
    S1 = O.Solution([[1, 0], [1, 1]], var_is_boson=[0, 1])
    beta = 3.0
    E = np.random.default_rng(6).uniform(-3, 3, (16, 2))
    # nu1 != nu2 in every row (Omega = 0 is a removable point of the bubble)
    X = np.array([[mats(2, beta), mats(0, beta)], [mats(-1, beta), mats(4, beta)]])
    v2, _, _ = S2.eval_energies(E, X, beta)
    v1, _, _ = S1.eval_energies(E, X[:, 0] - X[:, 1], beta)
    assert np.allclose(v2, v1, rtol=1e-13, atol=0)


def test_two_externals_conjugation_symmetry():
    """I(E, -X) = conj I(E, X) for imaginary external frequencies (every Matsubara set is symmetric
    under nu -> -nu and conj 1/(i w + E) = 1/(-i w + E)), checked with two externals on an
    order-3 self-energy diagram whose third internal variable is held external."""
    d = O.enumerate_sigma(3)[0]
    S = O.Solution(d["alpha"], eps=d["eps"], var_is_boson=[0, 0, 1, 0], n_ext=2)
    beta = 2.0
    E = np.random.default_rng(7).uniform(-2, 2, (8, d["alpha"].shape[0]))
    X = np.array([[mats(1, beta, boson=True), mats(0, beta)], [mats(-2, beta, boson=True), mats(2, beta)]])
    v, _, _ = S.eval_energies(E, X, beta)
    vc, _, _ = S.eval_energies(E, np.conj(X), beta)
    assert np.allclose(vc, np.conj(v), rtol=1e-12, atol=0)


BRUTE_EXT_CASES = [
    # (name, alpha, eps, boson, n_ext, beta, E, X row)
    ("two_fermionic_ext_m1", [[1, 1, 0], [1, 0, 1]], None, None, 2, 2.0, [0.4, -0.7], [mats(0, 2.0), mats(1, 2.0)]),
    ("bosonic_and_fermionic_ext_m1", [[1, 0, 0], [1, 1, 0], [1, 0, 1]], None, [0, 1, 0], 2, 1.5,
     [0.3, -0.8, 1.1], [mats(1, 1.5, boson=True), mats(-1, 1.5)]),
    ("three_ext_m1", [[1, 1, 0, 0], [1, 0, 1, 0], [1, 0, 0, 1]], None, [0, 1, 0, 0], 3, 2.0,
     [-0.5, 0.9, 0.25], [mats(2, 2.0, boson=True), mats(0, 2.0), mats(-3, 2.0)]),
    # order-2 self-energy with the transfer q held external: summed k', externals (q, k_ext)
    ("sigma2_q_external_m1", [[0, 1, 1], [1, 0, 0], [1, 1, 0]], None, [0, 1, 0], 2, 2.0, [0.8, -0.5, 0.45],
     [mats(1, 2.0, boson=True), mats(0, 2.0)]),
    # two internal sums, two externals (one bosonic), a double pole from equal labels
    ("double_pole_m2", [[1, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [-1, 1, 1, 1]],
     [[1, 0, 0, 0], [1, 0, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1]], [0, 0, 1, 0], 2, 2.0, [0.5, 0.0, -0.3, 0.9],
     [mats(1, 2.0, boson=True), mats(0, 2.0)]),
]


@pytest.mark.parametrize("case", BRUTE_EXT_CASES, ids=[c[0] for c in BRUTE_EXT_CASES])
def test_construction_with_several_externals_against_brute_force(case):
    """The AMI result with n_ext external frequencies equals the plain definition: truncated
    sums over the internal variables only (Eq. goal, externals fixed), with tail extrapolation;
    fermionic, bosonic and mixed externals, shift parities over several externals, a double pole."""
    name, alpha, eps, boson, n_ext, beta, E, X = case
    S = O.Solution(alpha, eps=eps, var_is_boson=boson, n_ext=n_ext)
    v, _, _ = S.eval_energies(np.array([E]), np.array([X]), beta)
    ref = extrapolated_sum(alpha, np.array(E, dtype=float), np.array(X), beta, n_ext, eps=eps, boson=boson)
    assert abs(v[0, 0] - ref) <= 1e-9 * abs(ref), (v[0, 0], ref)


def test_order3_sigma_with_held_external_variable_against_brute_force():
    """An order-3 self-energy diagram with its last internal variable held external (n_ext = 2,
    two sums left): the oracle's construction against the two-variable truncated sums."""
    d = O.enumerate_sigma(3)[0]
    alpha = d["alpha"]
    S = O.Solution(alpha, eps=d["eps"], var_is_boson=[0, 0, 1, 0], n_ext=2)
    beta = 1.5
    E = np.random.default_rng(8).uniform(-1.5, 1.5, alpha.shape[0])
    X = np.array([mats(1, beta, boson=True), mats(0, beta)])
    v, _, _ = S.eval_energies(E[None, :], X[None, :], beta)
    ref = extrapolated_sum(alpha, E, X, beta, 2, eps=d["eps"], boson=[0, 0, 1, 0])
    assert abs(v[0, 0] - ref) <= 1e-9 * abs(ref), (v[0, 0], ref)


def test_momentum_sampling_refuses_several_externals():
    """Momentum sampling (Sec. 5.2) appends one external momentum to the sampled ones, so the
    oracle's momentum mode takes n_ext = 1 only."""
    S = O.Solution([[1, 1, 0], [1, 0, 1]], n_ext=2)
    with pytest.raises(ValueError, match="one external momentum"):
        S.eval_momenta((1.0, 0.0, 0.0, 0.5, 0.5), 1, 0, 4, [1j], 2.0)

"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names the passage of arXiv:2311.17189 it checks, or the mathematics that fixes
the expected value: published known-answer vectors, closed forms derived by hand, the plain
definition of the Matsubara sum (brute force with tail extrapolation), symmetries of the
integrand, finite differences, and momentum conservation.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def f_fermi(beta, x):
    return 1.0 / (np.exp(beta * x) + 1.0)


def n_bose(beta, x):
    return 1.0 / (np.exp(beta * x) - 1.0)


def extrapolated_sum(alpha, E, X, beta, eps=None, boson=None, Ns=(62, 125, 250, 500, 1000, 2000)):
    """Plain definition (Eq. goal): truncated Matsubara sums on the box |n_l| <= N, extrapolated
    to N -> infinity.  A box cut through an absolutely convergent sum leaves a boundary error
    a/N + (b log N + c)/N^2 + (d log N + e)/N^3 + ...; fit those terms exactly on six boxes."""
    Ns = np.asarray(Ns, dtype=float)
    vals = np.array([O.brute_force(alpha, E, X, beta, int(N), eps=eps, var_is_boson=boson) for N in Ns])
    M = np.stack([np.ones_like(Ns), 1 / Ns, np.log(Ns) / Ns**2, 1 / Ns**2, np.log(Ns) / Ns**3, 1 / Ns**3], 1)
    return np.linalg.solve(M, vals)[0]


# ---------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors (Salmon et al., SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


# ---------------------------------------------------------------------------- trig
def test_sincos_against_high_precision():
    """The oracle's dispersion takes sin and cos from the C library (the paper leaves eps(k) to
    the user, Sec. 5.2): within one ulp of 50-digit values over the range of line momenta, exact
    at 0, and sin^2 + cos^2 = 1 as an identity that needs no reference."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    rng = np.random.default_rng(17)
    k = np.concatenate([rng.uniform(-7 * np.pi, 7 * np.pi, 4000), np.linspace(-22, 22, 1001),
                        np.array([np.pi / 2, np.pi, 1e-9, -3e-5])])
    s, c = O.sincos(k)
    for i in range(k.size):
        x = mpmath.mpf(float(k[i]))
        for got, ref in ((s[i], mpmath.sin(x)), (c[i], mpmath.cos(x))):
            r = float(ref)
            assert abs(got - r) <= np.spacing(abs(r)) + 1e-300, (k[i], got, r)
    s0, c0 = O.sincos([0.0])
    assert s0[0] == 0.0 and c0[0] == 1.0
    assert np.max(np.abs(s * s + c * c - 1.0)) < 5e-16


# ---------------------------------------------------------------------------- Fermi/Bose
@pytest.mark.parametrize("sigma", [1, -1])
@pytest.mark.parametrize("beta", [1.0, 8.0])
def test_fermi_value_and_first_derivative_closed_forms(sigma, beta):
    """g_sigma(x) = 1/(sigma e^{beta x} + 1): f for sigma=+1 and -n_B for sigma=-1 (Eq. Res_Th and
    the bosonic residue weight); first derivative -sigma beta e^{beta x}/(sigma e^{beta x}+1)^2."""
    for x in [-2.3, -0.7, -0.05, 0.03, 0.4, 1.9]:
        ex = math.exp(beta * x)
        g = 1.0 / (sigma * ex + 1.0)
        d1 = -sigma * beta * ex / (sigma * ex + 1.0) ** 2
        assert O.fermi_deriv(sigma, 0, beta, x) == pytest.approx(g, rel=1e-13)
        assert O.fermi_deriv(sigma, 1, beta, x) == pytest.approx(d1, rel=1e-12)
        if sigma == 1:
            assert O.fermi_deriv(1, 0, beta, x) == pytest.approx(f_fermi(beta, x), rel=1e-13)
        else:
            assert O.fermi_deriv(-1, 0, beta, x) == pytest.approx(-n_bose(beta, x), rel=1e-13)


@pytest.mark.parametrize("sigma", [1, -1])
@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_fermi_higher_derivatives_against_finite_differences(sigma, k):
    """d^k g/dx^k (the f^(m), b^(m) of multipole residues, Eq. Res_mul) against a 4th-order central
    difference of the (k-1)-th derivative."""
    beta = 2.0
    h = 1e-3
    for x in [-1.1, -0.4, 0.25, 0.9]:
        fd = (-O.fermi_deriv(sigma, k - 1, beta, x + 2 * h) + 8 * O.fermi_deriv(sigma, k - 1, beta, x + h)
              - 8 * O.fermi_deriv(sigma, k - 1, beta, x - h) + O.fermi_deriv(sigma, k - 1, beta, x - 2 * h)) / (12 * h)
        assert O.fermi_deriv(sigma, k, beta, x) == pytest.approx(fd, rel=2e-8, abs=1e-10)


def test_fermi_relative_accuracy_in_tails_and_near_zero():
    """g_sigma and its first derivatives keep full relative accuracy where they are tiny
    (beta x up to 600) and where the Bose form 1/(1 - e^{beta x}) cancels (beta x ~ 1e-9),
    compared with the definition evaluated in 60-digit arithmetic."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    for sigma in (1, -1):
        for bx in (-600.0, -75.0, -40.0, -12.0, -1e-3, -1e-9, 1e-9, 1e-3, 12.0, 40.0, 75.0, 600.0):
            beta = 2.0
            x = bx / beta
            e = mp.exp(mp.mpf(beta) * mp.mpf(x))
            g = 1 / (sigma * e + 1)
            d1 = -sigma * beta * e / (sigma * e + 1) ** 2
            assert O.fermi_deriv(sigma, 0, beta, x) == pytest.approx(float(g), rel=4e-15)
            assert O.fermi_deriv(sigma, 1, beta, x) == pytest.approx(float(d1), rel=1e-14)


def test_fermi_extreme_arguments_and_reflection():
    """No overflow at beta x = +-1000, and g_sigma(-x) = 1 - g_sigma(x) for both sigma."""
    for sigma in (1, -1):
        for x in (-1000.0, -50.0, 50.0, 1000.0):
            v = O.fermi_deriv(sigma, 0, 1.0, x)
            assert math.isfinite(v)
            for k in (1, 2, 3):
                assert math.isfinite(O.fermi_deriv(sigma, k, 1.0, x))
        for x in (0.3, 1.7, 25.0):
            assert O.fermi_deriv(sigma, 0, 3.0, -x) == pytest.approx(1.0 - O.fermi_deriv(sigma, 0, 3.0, x), rel=1e-14, abs=1e-300)
    assert O.fermi_deriv(1, 0, 1.0, 1000.0) == 0.0 or O.fermi_deriv(1, 0, 1.0, 1000.0) < 1e-300
    assert O.fermi_deriv(1, 0, 1.0, -1000.0) == 1.0


# ---------------------------------------------------------------------------- construction
PAPER_ALPHA = [[1, 0, 0], [0, 1, 0], [-1, 1, 1]]   # Sec. 5.1, the paper's order-2 example


def test_paper_example_closed_form():
    """Order-2 self-energy of Sec. 5.1 (alpha = (1,0,0), (0,1,0), (-1,1,1), eps = identity).
    Summing nu_1 then nu_2 by hand gives
    I = [f(-E1) - f(E3)] [f(-E2) + n_B(-E1-E3)] / (i nu + E1 + E3 - E2),
    a product of two two-leaf sums, the shape of the paper's Fig. treeflow."""
    S = O.Solution(PAPER_ALPHA)
    info = S.info()
    assert info["terms"] == 4 and info["fermi_factors"] == 8 and info["g_factors"] == 4
    rng = np.random.default_rng(1)
    for beta in (1.0, 3.0):
        E = rng.uniform(-4, 4, (20, 3))
        X = np.array([1j * np.pi / beta, 7j * np.pi / beta, -5j * np.pi / beta])
        v, _, _ = S.eval_energies(E, X, beta)
        for i in range(E.shape[0]):
            E1, E2, E3 = E[i]
            for fi, x in enumerate(X):
                cf = (f_fermi(beta, -E1) - f_fermi(beta, E3)) * (f_fermi(beta, -E2) + n_bose(beta, -E1 - E3)) / (x + E1 + E3 - E2)
                assert abs(v[fi, i] - cf) <= 1e-13 * abs(cf) + 1e-15


def test_bosonic_transfer_labelling_closed_form():
    """Order-2 Hubbard self-energy in the basis (q, k', k_ext) with lines q+k_ext, k', q+k' and q
    bosonic.  Summing q (weight -n_B) then k' by hand gives
    I = -[f(-E1) - f(-E3)] [f(-E2) + n_B(E1 - E3)] / (i nu + E1 + E2 - E3)."""
    S = O.Solution([[1, 0, 1], [0, 1, 0], [1, 1, 0]], var_is_boson=[1, 0, 0])
    assert S.info()["terms"] == 4
    rng = np.random.default_rng(2)
    beta = 5.0
    E = rng.uniform(-4, 4, (20, 3))
    X = np.array([1j * np.pi / beta, 3j * np.pi / beta])
    v, _, _ = S.eval_energies(E, X, beta)
    for i in range(E.shape[0]):
        E1, E2, E3 = E[i]
        for fi, x in enumerate(X):
            cf = -(f_fermi(beta, -E1) - f_fermi(beta, -E3)) * (f_fermi(beta, -E2) + n_bose(beta, E1 - E3)) / (x + E1 + E2 - E3)
            assert abs(v[fi, i] - cf) <= 1e-13 * abs(cf) + 1e-15


def test_closed_form_exact_arithmetic_wide_energies():
    """Against the same closed form evaluated in 50-digit arithmetic, over energies U(-8, 8) at
    beta=5 (Fermi tails down to e^-80, strong cancellation between terms): the error stays
    within 1e-13 of the rounding envelope sum_t |A| prod |FT factors| prod |G| on every sample."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    beta = 5.0
    S = O.Solution([[1, 0, 1], [0, 1, 0], [1, 1, 0]], var_is_boson=[1, 0, 0])
    E = np.random.default_rng(11).uniform(-8, 8, (300, 3))
    x = 1j * np.pi / beta
    v, _, env = S.eval_energies(E, [x], beta)
    f = lambda z: 1 / (mp.exp(beta * z) + 1)
    nb = lambda z: 1 / (mp.exp(beta * z) - 1)
    for i in range(E.shape[0]):
        E1, E2, E3 = (mp.mpf(float(e)) for e in E[i])
        ex = -(f(-E1) - f(-E3)) * (f(-E2) + nb(E1 - E3)) / (mp.mpc(0, x.imag) + E1 + E2 - E3)
        assert abs(v[0, i] - complex(ex)) <= 1e-13 * env[0, i]


def test_lindhard_bubble_closed_form():
    """Order 1 with a bosonic external frequency: (1/beta) sum_nu G(nu,E1) G(nu+Omega,E2)
    = [f(-E1) - f(-E2)] / (i Omega + E2 - E1)."""
    S = O.Solution([[1, 0], [1, 1]], var_is_boson=[0, 1])
    beta = 2.0
    E = np.array([[0.3, -0.9], [1.2, 2.5], [-3.0, 0.1]])
    X = np.array([2j * np.pi / beta, 6j * np.pi / beta])
    v, _, _ = S.eval_energies(E, X, beta)
    for i in range(E.shape[0]):
        E1, E2 = E[i]
        for fi, x in enumerate(X):
            cf = (f_fermi(beta, -E1) - f_fermi(beta, -E2)) / (x + E2 - E1)
            assert abs(v[fi, i] - cf) <= 1e-13 * abs(cf)


BRUTE_CASES = [
    # (name, alpha, eps, boson, beta, E, X)
    ("paper_order2_beta1", PAPER_ALPHA, None, None, 1.0, [2.1, 0.3, -1.1], 1j * np.pi),
    ("paper_order2_beta2", PAPER_ALPHA, None, None, 2.0, [0.7, -0.4, 1.3], 1j * np.pi / 2),
    ("paper_order2_beta5", PAPER_ALPHA, None, None, 5.0, [0.2, 0.35, -0.6], 3j * np.pi / 5),
    ("bosonic_q_order2", [[1, 0, 1], [0, 1, 0], [1, 1, 0]], None, [1, 0, 0], 2.0, [0.8, -0.5, 0.45], 1j * np.pi / 2),
    ("bubble_order1", [[1, 0], [1, 1]], None, [0, 1], 2.0, [0.3, -0.9], 2j * np.pi / 2),
    # double pole: lines 0 and 1 carry the same momentum and share one energy
    ("double_pole_order1", [[1, 0], [1, 0], [1, 1]], [[1, 0, 0], [1, 0, 0], [0, 0, 1]], [0, 1], 1.5,
     [0.6, 0.0, -0.8], 2j * np.pi / 1.5),
    ("triple_pole_order1", [[1, 0], [1, 0], [1, 0], [1, 1]],
     [[1, 0, 0, 0], [1, 0, 0, 0], [1, 0, 0, 0], [0, 0, 0, 1]], [0, 1], 1.5, [-0.45, 0.0, 0.0, 0.7], 4j * np.pi / 1.5),
    ("quadruple_pole_order1", [[1, 0], [1, 0], [1, 0], [1, 0], [1, 1]],
     [[1, 0, 0, 0, 0]] * 4 + [[0, 0, 0, 0, 1]], [0, 1], 1.2, [0.35, 0, 0, 0, -0.55], 2j * np.pi / 1.2),
    ("double_pole_order2", [[1, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 1, 1]],
     [[1, 0, 0, 0], [1, 0, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1]], None, 2.0, [0.5, 0.0, -0.3, 0.9], 1j * np.pi / 2),
]


@pytest.mark.parametrize("case", BRUTE_CASES, ids=[c[0] for c in BRUTE_CASES])
def test_construction_against_brute_force_matsubara_sums(case):
    """The AMI result equals the plain definition beta^-m sum_nu prod_j 1/(X_j + E_j) (Eq. goal)
    computed by truncated sums with tail extrapolation; covers fermionic and bosonic sums and
    poles of order 2, 3 and 4 (derivatives f', f'', f''' of Eq. Res_mul)."""
    name, alpha, eps, boson, beta, E, X = case
    S = O.Solution(alpha, eps=eps, var_is_boson=boson)
    v, _, _ = S.eval_energies(np.array([E]), [X], beta)
    ref = extrapolated_sum(alpha, np.array(E), X, beta, eps=eps, boson=boson)
    assert abs(v[0, 0] - ref) <= 1e-9 * abs(ref), (v[0, 0], ref)
    if "quadruple" in name:
        assert S.info()["max_der"] == 3


def test_symmetries_energy_reflection_and_conjugation():
    """I(-E, i nu) = (-1)^N conj I(E, i nu) and I(E, -i nu) = conj I(E, i nu), from
    conj 1/(i w + E) = 1/(-i w + E) and the symmetry of the Matsubara sets under nu -> -nu."""
    for alpha, boson in ((PAPER_ALPHA, None), ([[1, 0, 1], [0, 1, 0], [1, 1, 0]], [1, 0, 0])):
        S = O.Solution(alpha, var_is_boson=boson)
        N = len(alpha)
        beta = 3.0
        rng = np.random.default_rng(3)
        E = rng.uniform(-3, 3, (10, N))
        X = np.array([1j * np.pi / beta, 5j * np.pi / beta])
        v, _, _ = S.eval_energies(E, X, beta)
        vneg, _, _ = S.eval_energies(-E, X, beta)
        vconj, _, _ = S.eval_energies(E, np.conj(X), beta)
        assert np.allclose(vneg, (-1) ** N * np.conj(v), rtol=1e-12, atol=0)
        assert np.allclose(vconj, np.conj(v), rtol=1e-12, atol=0)


@pytest.mark.parametrize("order", [3, 4])
def test_integration_order_independence(order):
    """The Matsubara sums commute: summing the internal variables in reverse order gives a
    different term table but the same values (Sec. 5.1 fixes only the order 1 -> NINT).  The two
    tables form different energy combinations, whose rounding is amplified where a combination
    nearly cancels, so the bound is 1e-8 of the rounding envelope; an algebra mistake is O(1)."""
    d = O.enumerate_sigma(order)[0]
    S1 = O.Solution(d["alpha"], eps=d["eps"])
    S2 = O.Solution(d["alpha"], eps=d["eps"], order=list(range(order))[::-1])
    beta = 4.0
    E = O.sample_energies(d["alpha"], (1.0, -0.3, -0.5, np.pi / 2, np.pi / 2), 7, 0, 64)[0]
    X = np.array([1j * np.pi / beta, 3j * np.pi / beta])
    v1, _, en1 = S1.eval_energies(E, X, beta)
    v2, _, en2 = S2.eval_energies(E, X, beta)
    assert np.all(np.abs(v1 - v2) <= 1e-8 * np.maximum(en1, en2))


# ---------------------------------------------------------------------------- momenta
def test_momentum_composition_paper_example():
    """Line momenta K = k A^T with A = alpha (x) I_2 for the paper's worked example (Sec. 5.2):
    the printed A^T, applied to the sampled (k1, k2, q), must give the per-line dispersion the
    oracle uses.  Energies checked against numpy cos with the printed matrix."""
    AT = np.array([[1, 0, 0, 0, -1, 0], [0, 1, 0, 0, 0, -1], [0, 0, 1, 0, 1, 0],
                   [0, 0, 0, 1, 0, 1], [0, 0, 0, 0, 1, 0], [0, 0, 0, 0, 0, 1]], dtype=float)
    t, tp, mu, qx, qy = 1.0, -0.3, -0.5, 0.4, -1.2
    E, k = O.sample_energies(PAPER_ALPHA, (t, tp, mu, qx, qy), 99, 5, 1000)
    kk = np.concatenate([k.reshape(1000, 4), np.tile([qx, qy], (1000, 1))], 1)
    K = kk @ AT
    for j in range(3):
        kx, ky = K[:, 2 * j], K[:, 2 * j + 1]
        ref = mu + 2 * t * (np.cos(kx) + np.cos(ky)) + 4 * tp * np.cos(kx) * np.cos(ky)
        assert np.max(np.abs(E[:, j] - ref)) < 4e-15
    assert np.all(k >= -np.pi) and np.all(k < np.pi)


def test_momentum_samples_are_uniform():
    """The u -> k map over Philox words covers [-pi, pi) uniformly (mean 0, variance pi^2/3)."""
    _, k = O.sample_energies([[1, 0], [1, 1]], (1, 0, 0, 0, 0), 2023, 0, 200000)
    x = k.ravel()
    assert abs(x.mean()) < 0.02
    assert abs(x.var() - np.pi ** 2 / 3) < 0.03


# ---------------------------------------------------------------------------- derivatives
def test_dual_derivatives_against_finite_differences_energy_input():
    """Forward-mode dual numbers vs central differences along random energy and frequency
    directions, order-2 example with real-axis frequencies omega + i Gamma."""
    S = O.Solution(PAPER_ALPHA)
    rng = np.random.default_rng(4)
    E = rng.uniform(-3, 3, (8, 3))
    dE = rng.normal(size=(8, 3))
    X = np.array([0.3 + 0.05j, -1.1 + 0.05j])
    beta = 4.0
    h = 1e-5
    for dX in (0.0, 1.0):
        der = S.eval_energies_deriv(E, dE, X, dX, beta)
        vp, _, _ = S.eval_energies(E + h * dE, X + h * dX, beta)
        vm, _, _ = S.eval_energies(E - h * dE, X - h * dX, beta)
        fd = (vp - vm) / (2 * h)
        assert np.all(np.abs(der - fd) <= 1e-5 * np.abs(der) + 1e-7)


@pytest.mark.parametrize("which", ["omega", "mu", "kx", "ky"])
def test_dual_derivatives_against_finite_differences_momentum(which):
    """d Sigma/d omega, d/d mu, d/d k_ext through the momentum path (dispersion gradient
    included) vs central differences of the oracle's own values."""
    d = O.enumerate_sigma(3)[0]
    S = O.Solution(d["alpha"], eps=d["eps"])
    lat = np.array([1.0, -0.3, -0.2, np.pi / 2, np.pi / 3])
    beta = 3.0
    X = np.array([0.4 + 0.3j, -0.9 + 0.3j])
    h = 1e-5
    n = 16
    _, der = S.eval_momenta_deriv(lat, 11, 0, n, X, beta, which)
    lp, lm = lat.copy(), lat.copy()
    Xp, Xm = X.copy(), X.copy()
    if which == "omega":
        Xp = X + h; Xm = X - h
    else:
        idx = {"mu": 2, "kx": 3, "ky": 4}[which]
        lp[idx] += h; lm[idx] -= h
    vp = S.eval_momenta(lp, 11, 0, n, Xp, beta)["values"]
    vm = S.eval_momenta(lm, 11, 0, n, Xm, beta)["values"]
    fd = (vp - vm) / (2 * h)
    scale = np.abs(der) + np.abs(fd)
    assert np.all(np.abs(der - fd) <= 1e-5 * scale + 1e-8), np.max(np.abs(der - fd) / scale)


# ---------------------------------------------------------------------------- enumerator
@pytest.mark.parametrize("order", [2, 3, 4, 5])
def test_enumerated_labels_conserve_momentum(order):
    """Every enumerated diagram is labelled with alpha in {-1,0,1}, N = 2m-1 lines, m loop
    variables, and conserves momentum at every interaction (Sec. 2.5: momentum-conserving
    labels).  Rebuild the graph from the canonical code and check in = out at each node."""
    ds = O.enumerate_sigma(order)
    m = order
    for d in ds:
        a = d["alpha"]
        assert a.shape == (2 * m - 1, m + 1)
        assert np.all(np.abs(a) <= 1)
        code = d["code"]
        pu = [None] * (m + 1)
        pd = [None] * m
        pu[m] = code[0]
        for c in range(m):
            pu[c] = code[1 + 2 * c]
            pd[c] = code[2 + 2 * c]
        lines = [(c, pu[c]) for c in range(m) if pu[c] != m] + [(c, pd[c]) for c in range(m)]
        ext = np.zeros(m + 1, dtype=int)
        ext[m] = 1
        for node in range(m):
            tot = np.zeros(m + 1, dtype=int)
            for j, (s, t) in enumerate(lines):
                if t == node:
                    tot += a[j]
                if s == node:
                    tot -= a[j]
            if pu[m] == node:
                tot += ext
            if pu[node] == m:
                tot -= ext
            assert np.all(tot == 0)
        # every loop variable is carried somewhere; each line carries a loop momentum (1PI)
        assert np.all(np.any(a[:, :m] != 0, axis=1))
        # equal labels share one base energy
        rep = d["eps"].argmax(1)
        for j in range(a.shape[0]):
            assert np.array_equal(a[j], a[rep[j]])


def test_enumerator_counts_and_order2_structure():
    """Hubbard self-energy diagrams without tadpoles: one diagram at order 2, with one closed
    loop (sign -1) and three lines.  Counts at orders 3-5 are recorded for the cross-check
    against the library's enumerator (parity unpinned beyond that cross-check)."""
    d2 = O.enumerate_sigma(2)
    assert len(d2) == 1 and d2[0]["loops"] == 1 and d2[0]["sign"] == -1.0
    assert [len(O.enumerate_sigma(m)) for m in (1, 2, 3, 4, 5)] == [0, 1, 2, 12, 70]


def test_enumerated_order2_matches_second_order_sigma_mean():
    """The order-2 diagram from the enumerator and the hand-labelled order-2 self-energy are the
    same integral: their Monte Carlo means over independent samples agree within 5 sigma."""
    d = O.enumerate_sigma(2)[0]
    S1 = O.Solution(d["alpha"], eps=d["eps"])
    S2 = O.Solution([[1, 0, 1], [0, 1, 0], [1, 1, 0]], var_is_boson=[1, 0, 0])
    lat = (1.0, 0.0, 0.0, np.pi / 2, np.pi / 2)
    beta = 2.0
    X = [1j * np.pi / beta]
    n = 100000
    r1 = S1.eval_momenta(lat, 5, 0, n, X, beta, per_sample=False, threads=4)
    r2 = S2.eval_momenta(lat, 6, 0, n, X, beta, per_sample=False, threads=4)
    se = np.sqrt((r1["var"][0] + r2["var"][0]) / n)
    diff = r1["mean"][0] - r2["mean"][0]
    assert abs(diff.real) < 5 * se[0] and abs(diff.imag) < 5 * se[1]


# ---------------------------------------------------------------------------- sensitivities
SENS_CASES = [
    ("paper_order2", [[1, 0, 0], [0, 1, 0], [-1, 1, 1]], None, None, 2.0),
    ("bosonic_q_order2", [[1, 0, 1], [0, 1, 0], [1, 1, 0]], None, [1, 0, 0], 5.0),
    ("quadruple_pole", [[1, 0], [1, 0], [1, 0], [1, 0], [1, 1]], [[1, 0, 0, 0, 0]] * 4 + [[0, 0, 0, 0, 1]],
     [0, 1], 1.2),
]


@pytest.mark.parametrize("case", SENS_CASES, ids=[c[0] for c in SENS_CASES])
def test_energy_sensitivity_bounds_gradient_and_finite_changes(case):
    """The oracle's energy sensitivity sum_t sum_j |d term_t / d E_j| is an upper bound of what a
    change of the base energies can do to the value, the quantity the GPU parity tests use to
    allow for the two sides' different cos/sin: (i) it is at least sum_j |d Sigma / d E_j|, from
    dual numbers along each coordinate; (ii) moving every energy by at most h (random signs)
    changes the value by at most h sens (first order; h small); (iii) it is exact where the
    solution is one factor of one energy: the double pole sum_nu 1/(i nu + E)^2 / beta leaves a
    single term A f'(E), whose sensitivity is |A f''(E)| = |d Sigma / d E|."""
    _, alpha, eps, boson, beta = case
    S = O.Solution(alpha, eps=eps, var_is_boson=boson)
    rng = np.random.default_rng(5)
    N = np.asarray(alpha).shape[0]
    E = rng.uniform(-2, 2, (6, N))
    X = np.array([1j * np.pi / beta, 0.7 + 0.1j])
    v, _, env, sens = S.eval_energies(E, X, beta, sens=True)
    grad = np.zeros_like(sens)
    for j in range(N):
        dE = np.zeros_like(E)
        dE[:, j] = 1.0
        grad += np.abs(S.eval_energies_deriv(E, dE, X, 0.0, beta))
    assert np.all(grad <= sens * (1 + 1e-12)), np.max(grad / sens)
    h = 1e-7
    for _ in range(4):
        dE = h * rng.choice([-1.0, 1.0], size=E.shape)
        vp, _, _ = S.eval_energies(E + dE, X, beta)
        assert np.all(np.abs(vp - v) <= h * sens * (1 + 1e-4) + 1e-13 * env)
    # double pole: one term A f'(E) of one energy, where the bound is attained
    P = O.Solution([[1, 0], [1, 0]], eps=[[1, 0], [1, 0]])
    assert P.info()["terms"] == 1
    E1 = np.array([[0.3, 0.0], [-1.7, 0.0], [0.05, 0.0]])
    X1 = np.array([0.0j])
    _, _, _, s1 = P.eval_energies(E1, X1, beta, sens=True)
    dE = np.zeros_like(E1)
    dE[:, 0] = 1.0
    g1 = np.abs(P.eval_energies_deriv(E1, dE, X1, 0.0, beta))
    assert np.allclose(s1, g1, rtol=1e-13, atol=0)


@pytest.mark.parametrize("case", SENS_CASES, ids=[c[0] for c in SENS_CASES])
def test_derivative_sensitivity_bounds_second_differences(case):
    """The derivative's energy sensitivity sum_t sum_j |d (d term_t) / d E_j| bounds
    sum_j |d D / d E_j| for D = d Sigma / d mu (every base energy moves with mu) and for
    D = d Sigma / d omega, with d D / d E_j from central differences of the dual derivative."""
    _, alpha, eps, boson, beta = case
    S = O.Solution(alpha, eps=eps, var_is_boson=boson)
    rng = np.random.default_rng(9)
    N = np.asarray(alpha).shape[0]
    E = rng.uniform(-2, 2, (5, N))
    X = np.array([1j * np.pi / beta, 0.4 + 0.2j])
    h = 1e-6
    for dE_dir, dX in ((np.ones_like(E), 0.0), (np.zeros_like(E), 1.0)):
        _, dsens = S.eval_energies_deriv(E, dE_dir, X, dX, beta, sens=True)
        tot = np.zeros_like(dsens)
        for j in range(N):
            e = np.zeros_like(E)
            e[:, j] = h
            tot += np.abs(S.eval_energies_deriv(E + e, dE_dir, X, dX, beta)
                          - S.eval_energies_deriv(E - e, dE_dir, X, dX, beta)) / (2 * h)
        assert np.all(tot <= dsens * (1 + 1e-5) + 1e-9), np.max(tot / dsens)


def test_monte_carlo_mean_and_variance_are_numpy_moments():
    """The oracle's Monte Carlo reduction (Sec. 2.3, "summing the rows"; variance unbiased, n - 1)
    against numpy's mean and var(ddof=1) of the oracle's own per-sample values, for Re and Im,
    at a sample count where dividing by n instead of n - 1 would differ by 2 %."""
    d = O.enumerate_sigma(3)[1]
    S = O.Solution(d["alpha"], eps=d["eps"])
    lat = (1.0, -0.3, -0.5, np.pi / 2, np.pi / 2)
    X = 1j * np.pi / 8.0 * np.array([1, 3, 5])
    for n in (2, 50, 3001):
        r = S.eval_momenta(lat, 42, 7, n, X, 8.0, per_sample=True)
        v = r["values"]
        scale = np.mean(np.abs(v), axis=1)
        assert np.all(np.abs(r["mean"] - v.mean(axis=1)) <= 1e-14 * scale)
        for part, k in ((np.real, 0), (np.imag, 1)):
            ref = np.var(part(v), axis=1, ddof=1)
            assert np.all(np.abs(r["var"][:, k] - ref) <= 1e-12 * ref), (n, k)
    r1 = S.eval_momenta(lat, 42, 7, 1, X, 8.0, per_sample=True)
    assert np.array_equal(r1["mean"], r1["values"][:, 0]) and np.all(r1["var"] == 0.0)

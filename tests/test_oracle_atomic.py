"""A pin of the enumerated self-energy diagrams (set, signs and prefactors) from physics, outside
both enumerators: the half-filled Hubbard atom.

With t = t' = 0 and particle-hole symmetry (every line energy 0), the exact self-energy of the
single-site Hubbard model at half filling is Sigma(i omega) = U/2 + U^2 / (4 i omega) at every
temperature.  It is a polynomial in U, and the tadpole-free expansion (the Hartree term U/2 is
absorbed in the chemical potential, exactly, since the density stays 1/2 per spin) must reproduce
its Taylor coefficients order by order: the order-2 diagram sums to U^2 / (4 i omega) and the
diagrams of every order n >= 3 sum to zero.  A missing, duplicated or sign-flipped diagram leaves
a remainder of the size of that diagram.

The symbolic solutions have degenerate poles at zero energy, so the limit is approached: each
diagram gets base energies delta * r (one fixed random direction r per diagram) and the order sum
S(delta) must vanish as delta -> 0.  At orders 2-4 it vanishes linearly (halving delta halves
it) and the linear (Richardson) extrapolation 2 S(delta / 2) - S(delta) lies far below the
smallest diagram of the order, so a single wrong diagram would show.  At order 5 the cancellation
between terms grows like delta^-(m-1) and reaches the rounding floor below delta ~ 0.05; there
the sum is checked to fall towards zero (at least linearly in delta) to a few per cent of
the largest diagram, which catches an error in any diagram above that size but not in the
smallest ones (some are 1e-3 of the largest)."""
import math

import numpy as np
import pytest

import oracle as O

BETA = 2.0
X = np.array([1j * math.pi / BETA, 3j * math.pi / BETA, 7j * math.pi / BETA])


def order_values(m, deltas):
    """Per diagram of order m, its value (sign and prefactor included) at base energies
    delta * r for each delta: {delta: [n_diagrams, n_f]}."""
    rng = np.random.default_rng(100 + m)
    sols = []
    for d in O.enumerate_sigma(m):
        pre = (-1.0) ** m * (-1.0) ** d["loops"]
        nb = np.asarray(d["eps"]).shape[1]
        sols.append((O.Solution(d["alpha"], eps=d["eps"], prefactor=pre), rng.uniform(-1.0, 1.0, size=(1, nb))))
    return {dl: np.array([sol.eval_energies(dl * r, X, BETA)[0][:, 0] for sol, r in sols]) for dl in deltas}


@pytest.mark.parametrize("m", [2, 3, 4])
def test_orders_2_to_4_reach_the_atomic_self_energy(m):
    d1, d2 = 0.02, 0.01
    v = order_values(m, (d1, d2))
    exact = 1.0 / (4.0 * X) if m == 2 else np.zeros(len(X))      # U = 1
    s1, s2 = v[d1].sum(axis=0) - exact, v[d2].sum(axis=0) - exact
    ratio = np.abs(s2) / np.abs(s1)
    assert np.all((ratio > 0.45) & (ratio < 0.55)), ratio          # linear approach
    extrap = np.abs(2.0 * s2 - s1)
    smallest = np.min(np.abs(v[d2]), axis=0)
    assert np.all(extrap <= 0.25 * smallest), (extrap, smallest)


def test_order_5_sum_falls_towards_zero():
    v = order_values(5, (0.32, 0.16, 0.08))
    s = {dl: np.abs(v[dl].sum(axis=0)) for dl in v}
    largest = np.max(np.abs(v[0.08]))
    assert np.all(s[0.16] <= 0.55 * s[0.32]) and np.all(s[0.08] <= 0.55 * s[0.16]), s
    assert np.all(s[0.08] <= 0.05 * largest), (s[0.08], largest)


def test_a_sign_flipped_diagram_is_caught():
    """The check of orders 2-4 above, applied with one order-4 diagram's sign flipped (a mistake
    planted in the values, on the CPU): the remainder no longer vanishes."""
    d1, d2 = 0.02, 0.01
    v = order_values(4, (d1, d2))
    smallest = np.min(np.abs(v[d2]), axis=0)
    k = int(np.argmin(np.abs(v[d2][:, 0])))                         # the hardest one to see
    for dl in v:
        v[dl][k] *= -1.0
    extrap = np.abs(2.0 * v[d2].sum(axis=0) - v[d1].sum(axis=0))
    assert np.any(extrap > 0.25 * smallest)

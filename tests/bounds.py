"""Per-sample parity bounds of the momentum-mode GPU tests (helper module, not a test file).

The kernels and the CPU oracle draw the same Philox momenta and form the same line momenta bit
for bit.  The dispersion eps(k) is the user's (Sec. 5.2), and the two sides evaluate it
differently: the oracle with the C library's cos/sin and a plain formula, the kernels with their
own Cody-Waite cos/sin (pinned against the C library to TRIG_ERR in tests/test_gpu_math.py) and
an fma formula.  So their base energies differ by at most

    dE = (4|t| + 8|t'|) TRIG_ERR + 8u (|mu| + 4|t| + 4|t'|)

(E = mu + 2t(cx + cy) + 4t' cx cy: each cosine moves by at most TRIG_ERR, and each side rounds
at most four times on quantities no larger than |mu| + 4|t| + 4|t'|), and the slopes
dE/dk = -(2t + 4t' cos k_perp) sin k that the adjoint uses for k_ext by at most

    dG = (2|t| + 8|t'|) TRIG_ERR + 8u (2|t| + 4|t'|).

A difference dE in every base energy moves a value by at most dE * sens to first order, sens =
sum_t sum_j |d term_t / d E_j| from the oracle (pinned in tests/test_oracle_pins.py).  The
per-sample bound is therefore the rounding part RTOL * envelope (the relative 1e-11 of the
target, scaled to the terms that cancel) plus twice that first-order input part; for a
derivative, RTOL * derivative envelope plus twice (dE * dsens + dG * sens), the slope term only
for the k_ext directions.  With energy input both sides read the same energies and only the
rounding part applies.
"""
import numpy as np

RTOL = 1e-11
U = 2.0 ** -53
TRIG_ERR = 3e-16


def energy_error(lat):
    t, tp, mu = abs(lat[0]), abs(lat[1]), abs(lat[2])
    return (4 * t + 8 * tp) * TRIG_ERR + 8 * U * (mu + 4 * t + 4 * tp)


def slope_error(lat):
    t, tp = abs(lat[0]), abs(lat[1])
    return (2 * t + 8 * tp) * TRIG_ERR + 8 * U * (2 * t + 4 * tp)


def value_pert(ref, lat):
    """Input part of the per-sample value bound: twice dE times the oracle's sensitivity."""
    return 2.0 * energy_error(lat) * ref["sens"]


def value_bound(ref, lat):
    return RTOL * ref["envelope"] + value_pert(ref, lat)


def deriv_bound(lat, which, denv, dsens, sens):
    """Per-sample bound on a derivative along which in {'omega', 'mu', 'kx', 'ky'}."""
    pert = energy_error(lat) * dsens
    if which in ("kx", "ky"):
        pert = pert + slope_error(lat) * sens
    return RTOL * denv + 2.0 * pert


def oracle_deriv(S, lat, seed, off, n, X, beta, which, threads=8):
    """(derivative [n_f, n], per-sample bound [n_f, n]) from the oracle's dual numbers."""
    _, der, denv, dsens, sens = S.eval_momenta_deriv(lat, seed, off, n, X, beta, which, threads=threads,
                                                     sens=True)
    return der, deriv_bound(lat, which, denv, dsens, sens)


def mean_scale(ref, lat):
    """Bound scale of a Monte Carlo mean: the mean of the per-sample bounds over RTOL plus the mean
    |value| (the summation's own rounding)."""
    return np.mean(value_bound(ref, lat), axis=1) / RTOL + np.mean(np.abs(ref["values"]), axis=1)

"""Seeded synthetic workloads: parameters and input generators only.

This module holds none of the method's arithmetic.  It names the problem instances (lattice
parameters, temperatures, external frequencies, seeds, sample counts) and generates the
random inputs that are passed to both the CUDA path and the CPU oracle.  Momentum samples are
not generated here: each side draws them from Philox4x32-10 (Salmon et al., SC'11) with the
counter layout (sample_lo, sample_hi, internal_variable, 0) and key (seed_lo, seed_hi).

The paper's benchmark diagrams (its Fig. diagrams) are not available, so the instances below
use Hubbard self-energy diagrams from this project's own enumerator at the paper's orders.
"""
import math

import numpy as np

PI = math.pi
SEED = 20231128


def matsubara(beta, n_freq, first=0):
    """Fermionic Matsubara frequencies i(2n+1)pi/beta, n = first .. first+n_freq-1
    (the paper's example frequencies, Sec. 5.1)."""
    n = np.arange(first, first + n_freq, dtype=np.float64)
    return 1j * (2.0 * n + 1.0) * PI / beta


def real_axis(omega_lo, omega_hi, n, gamma):
    """omega + i Gamma on a uniform grid (analytic continuation i nu -> omega + i0+)."""
    return np.linspace(omega_lo, omega_hi, n) + 1j * gamma


# Order-2 Hubbard self-energy in the basis (q, k', k_ext): lines q+k_ext, k', q+k'; q is a
# bosonic transfer, k' fermionic.  t=1, mu=0, beta=5, U=1, one frequency i pi/beta, 1e5 samples.
ORDER2 = dict(
    name="order2_hubbard_sigma",
    alpha=np.array([[1, 0, 1], [0, 1, 0], [1, 1, 0]], dtype=np.int32),
    var_is_boson=np.array([1, 0, 0], dtype=np.int32),
    t=1.0, tp=0.0, mu=0.0, beta=5.0, U=1.0, kext=(PI / 2, PI / 2),
    n_freq=1, n_samples=100_000, seed=SEED,
)

# Order-4 Hubbard self-energy: the diagram with the largest flat term count among the order-4
# diagrams of the project's enumerator (canonical code below; 7 lines, 4 loop momenta).
# t=1, t'=-0.3, mu=-0.5, beta=8, 16 fermionic Matsubara frequencies n=0..15, 2^24 samples.
ORDER4 = dict(
    name="order4_hubbard_sigma",
    order=4,
    code=(0, 1, 1, 4, 2, 3, 3, 2, 0),
    t=1.0, tp=-0.3, mu=-0.5, beta=8.0, U=1.0, kext=(PI / 2, PI / 2),
    n_freq=16, n_samples=1 << 24, seed=SEED,
)

# Order-3 self-energy continued to the real axis: omega + i 0.05 on 256 points in [-4, 4].
ORDER3_REAL = dict(
    name="order3_sigma_real_axis",
    order=3, diagram_index=0,
    t=1.0, tp=0.0, mu=0.0, beta=10.0, U=1.0, kext=(PI / 2, PI / 2),
    omega=(-4.0, 4.0, 256), gamma=0.05, n_samples=1 << 22, seed=SEED,
)

# Large order: the order-5 diagram with the largest flat term table among the project's
# enumerated order-5 diagrams (744 terms; lowest enumeration index among equals; the multipole
# residues there need Fermi derivatives up to first order).  t=1, t'=0, mu=0, one frequency
# i pi/beta, 2^26 samples at each beta in (2, 5, 10, 20); forward and adjoint.
ORDER5 = dict(
    name="order5_hubbard_sigma",
    order=5,
    code=(0, 1, 1, 5, 2, 3, 3, 4, 4, 2, 0),
    t=1.0, tp=0.0, mu=0.0, betas=(2.0, 5.0, 10.0, 20.0), U=1.0, kext=(PI / 2, PI / 2),
    n_freq=1, n_samples=1 << 26, seed=SEED,
)

# Order 6 (the paper's scaling study runs to orders 6 and 9, Sec. 6.2): the order-6 diagram with
# the largest flat table of this enumerator (5136 terms), forward + adjoint over 2^24 samples at
# the order-5 workload's temperatures, one frequency i pi/beta.
ORDER6 = dict(
    name="order6_hubbard_sigma",
    order=6,
    code=(0, 1, 1, 6, 2, 4, 3, 5, 0, 3, 5, 2, 4),
    t=1.0, tp=0.0, mu=0.0, betas=(2.0, 5.0, 10.0, 20.0), U=1.0, kext=(PI / 2, PI / 2),
    n_freq=1, n_samples=1 << 24, seed=SEED,
)

# The paper's evaluation example at its own size (Sec. 5.1): the order-2 integrand of Sec. 5
# (frequency labels (1,0,0), (0,1,0), (-1,1,1), identity energies) on 10^6 rows of energies
# uniform on (-8, 8) and 100 fermionic Matsubara frequencies, beta = 1.
ENERGY_X1 = dict(
    name="energy_input_order2_x1",
    alpha=np.array([[1, 0, 0], [0, 1, 0], [-1, 1, 1]], dtype=np.int32),
    a=8.0, beta=1.0, n_freq=100, n_e=1_000_000, seed=SEED,
)

# Several external frequencies (Sec. 2.3: frequency_t rows with m + n_nu entries, n_nu > 1): the
# order-4 diagram of ORDER4 with its last loop frequency held external beside the external one
# (two fermionic externals nu', nu; three sums left), on energy input like the paper's example:
# 10^6 rows of energies uniform on (-8, 8), 100 frequency rows (nu'_{n'}, nu_n) on the 10 x 10
# grid n', n = 0..9, beta = 1.
TWO_FREQ_X1 = dict(
    name="order4_two_external_x1",
    order=4, code=(0, 1, 1, 4, 2, 3, 3, 2, 0), held=3,
    a=8.0, beta=1.0, n_grid=10, n_e=1_000_000, seed=SEED,
)


def hold_external(alpha, held):
    """Labels with internal variable `held` moved to the external block: columns reordered so the
    other internal variables come first, then `held`, then the original external (n_ext = 2)."""
    alpha = np.asarray(alpha)
    m = alpha.shape[1] - 1
    cols = [l for l in range(m) if l != held] + [held, m]
    return np.ascontiguousarray(alpha[:, cols])


def matsubara_grid(beta, n1, n2):
    """Rows (i nu'_{n'}, i nu_n), n' = 0..n1-1 (slow), n = 0..n2-1 (fast), both fermionic."""
    a, b = np.meshgrid(matsubara(beta, n1), matsubara(beta, n2), indexing="ij")
    return np.stack([a.ravel(), b.ravel()], axis=1)


# Every order-2..5 diagram in one launch: diagram d gets 2^(20 + d mod 4) samples, 32 freqs.
ALL_ORDERS = dict(
    name="sigma_orders_2_to_5",
    orders=(2, 3, 4, 5), t=1.0, tp=0.0, mu=0.0, beta=5.0, U=1.0, kext=(PI / 2, PI / 2),
    n_freq=32, seed=SEED,
)


def all_orders_samples(d):
    return 1 << (20 + d % 4)


def lattice(cfg):
    """(t, t', mu, kx_ext, ky_ext) as passed to both sides."""
    return (cfg["t"], cfg["tp"], cfg["mu"], cfg["kext"][0], cfg["kext"][1])


def random_energies(n_e, n_lines, a=8.0, seed=SEED):
    """Energy-input workload of the paper's evaluation example (Sec. 5.1): base energies
    uniform on (-a, a), one row per configuration."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-a, a, size=(n_e, n_lines))

"""Host-side Monte Carlo bookkeeping: sharding of the sample stream across ranks and the
merge of per-shard means and variances.

Samples are independent, so ranks take disjoint Philox counter ranges and need no data
exchange; their {count, mean, M2} statistics merge exactly with the pairwise update of
Chan, Golub and LeVeque (1979).
"""
import numpy as np


def shard(rank, world, n_per_rank, base_offset=0):
    """Counter offset and count of rank `rank`: ranks own consecutive blocks of n_per_rank."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return base_offset + rank * n_per_rank, n_per_rank


def merge(stats):
    """stats: iterable of (n, mean complex [n_f], var float [n_f, 2]) with unbiased variances of
    Re and Im.  Returns the same triple for the union of the samples."""
    it = iter(stats)
    n, mean, var = next(it)
    mean = np.asarray(mean, dtype=np.complex128).copy()
    m2 = np.asarray(var, dtype=np.float64) * max(n - 1, 0)
    for nb, mb, vb in it:
        mb = np.asarray(mb, dtype=np.complex128)
        m2b = np.asarray(vb, dtype=np.float64) * max(nb - 1, 0)
        tot = n + nb
        d = mb - mean
        mean = mean + d * (nb / tot)
        dd = np.stack([d.real, d.imag], axis=-1)
        m2 = m2 + m2b + dd * dd * (n * nb / tot)
        n = tot
    return n, mean, m2 / max(n - 1, 1)

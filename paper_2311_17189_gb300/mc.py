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


class Accumulator:
    """Monte Carlo state of one evaluation that grows chunk by chunk, so that a run can stop and
    resume: the merged {n, mean, var} per frequency and the next Philox counter offset.  Chunks
    are merged in order with merge(), and the state is saved without rounding (hex floats), so
    chunks c1..ck give the same bits whether they run in one process or across save() and load()."""

    def __init__(self, n_f, seed, offset=0):
        self.n_f, self.seed, self.offset = int(n_f), int(seed), int(offset)
        self.n = 0
        self.mean = np.zeros(self.n_f, dtype=np.complex128)
        self.var = np.zeros((self.n_f, 2), dtype=np.float64)

    def add(self, n, mean, var):
        """Merge the statistics of the next n samples of the stream (counters offset .. offset+n-1)."""
        mean = np.asarray(mean, dtype=np.complex128).reshape(self.n_f)
        var = np.asarray(var, dtype=np.float64).reshape(self.n_f, 2)
        if self.n == 0:
            self.n, self.mean, self.var = int(n), mean.copy(), var.copy()
        else:
            self.n, self.mean, self.var = merge([(self.n, self.mean, self.var), (int(n), mean, var)])
        self.offset += int(n)
        return self

    def run(self, diagram, lattice, X, beta, n_chunk, chunks=1):
        """Evaluate `chunks` more chunks of n_chunk samples with tami_forward and merge them."""
        for _ in range(int(chunks)):
            mean, var, _ = diagram.forward(lattice, self.seed, self.offset, n_chunk, X, beta)
            self.add(n_chunk, mean.cpu().numpy(), var.cpu().numpy())
        return self

    def state(self):
        h = lambda a: [float(v).hex() for v in np.ravel(a)]
        return {"n_f": self.n_f, "seed": self.seed, "offset": self.offset, "n": self.n,
                "mean_re": h(self.mean.real), "mean_im": h(self.mean.imag), "var": h(self.var)}

    def save(self, path):
        import json
        with open(path, "w") as f:
            json.dump(self.state(), f)

    @classmethod
    def load(cls, path):
        import json
        with open(path) as f:
            s = json.load(f)
        a = cls(s["n_f"], s["seed"], s["offset"])
        a.n = int(s["n"])
        u = lambda v: np.array([float.fromhex(x) for x in v], dtype=np.float64)
        a.mean = np.empty(a.n_f, dtype=np.complex128)
        a.mean.real, a.mean.imag = u(s["mean_re"]), u(s["mean_im"])
        a.var = u(s["var"]).reshape(a.n_f, 2)
        return a

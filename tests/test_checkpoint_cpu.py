"""Checkpoint and resume of the Monte Carlo state (mc.Accumulator), on CPU with synthetic chunk
statistics: the saved state round-trips exactly, chunks merged across a save and a load give the
same bits as the same chunks merged in one go, and the merged statistics are those of the union
of the samples (numpy mean and unbiased variance of the concatenation)."""
import numpy as np

from paper_2311_17189_gb300 import mc


def chunk_stats(x):
    """(n, mean, var) of complex samples x [n_f, n] as the forward kernel reports them."""
    return x.shape[1], x.mean(axis=1), np.stack([x.real.var(axis=1, ddof=1), x.imag.var(axis=1, ddof=1)], axis=-1)


def test_resume_is_bitwise_and_statistics_are_exact(tmp_path):
    rng = np.random.default_rng(5)
    n_f, sizes = 3, [1000, 777, 1000, 64, 5]
    chunks = [rng.normal(1.5, 2.0, (n_f, k)) + 1j * rng.normal(-0.5, 0.3, (n_f, k)) for k in sizes]
    one = mc.Accumulator(n_f, seed=7)
    for x in chunks:
        one.add(*chunk_stats(x))
    part = mc.Accumulator(n_f, seed=7)
    for x in chunks[:2]:
        part.add(*chunk_stats(x))
    path = tmp_path / "state.json"
    part.save(path)
    resumed = mc.Accumulator.load(path)
    assert resumed.state() == part.state()
    for x in chunks[2:]:
        resumed.add(*chunk_stats(x))
    assert resumed.offset == one.offset == sum(sizes)
    assert resumed.n == one.n
    assert np.array_equal(resumed.mean.view(np.uint64), one.mean.view(np.uint64))
    assert np.array_equal(resumed.var.view(np.uint64), one.var.view(np.uint64))
    allx = np.concatenate(chunks, axis=1)
    n, m, v = chunk_stats(allx)
    assert one.n == n
    assert np.allclose(one.mean, m, rtol=1e-14, atol=0)
    assert np.allclose(one.var, v, rtol=1e-12, atol=0)

"""Checkpoint and resume with the GPU forward: four chunks of the order-4 workload's stream merged
in one process equal, bit for bit, two chunks saved to a file, loaded and continued by two more;
and the merged mean agrees with one launch over the same samples (which groups the partial sums
differently)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import mc
from paper_2311_17189_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_checkpoint_resume_equals_an_uninterrupted_run(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    c = W.ORDER4
    d = next(x for x in T.enumerate_sigma(4) if tuple(x["code"]) == c["code"])
    D = T.Diagram(d["alpha"], eps=d["eps"]).upload(0)
    X, lat, beta, k = W.matsubara(c["beta"], c["n_freq"]), W.lattice(c), c["beta"], 1 << 16
    one = mc.Accumulator(len(X), c["seed"]).run(D, lat, X, beta, k, chunks=4)
    part = mc.Accumulator(len(X), c["seed"]).run(D, lat, X, beta, k, chunks=2)
    path = tmp_path / "mc_state.json"
    part.save(path)
    resumed = mc.Accumulator.load(path).run(D, lat, X, beta, k, chunks=2)
    assert resumed.offset == one.offset == 4 * k and resumed.n == one.n == 4 * k
    assert np.array_equal(resumed.mean.view(np.uint64), one.mean.view(np.uint64))
    assert np.array_equal(resumed.var.view(np.uint64), one.var.view(np.uint64))
    mean, var, ps = D.forward(lat, c["seed"], 0, 4 * k, X, beta, per_sample=True)
    scale = ps.abs().mean(dim=1).cpu().numpy()
    assert np.all(np.abs(mean.cpu().numpy() - one.mean) <= 1e-12 * scale)
    assert np.allclose(var.cpu().numpy(), one.var, rtol=1e-10, atol=0)

"""The N>1 path on CPU: two gloo ranks take disjoint blocks of the Philox sample stream
(mc.shard), evaluate their shard (here with the CPU oracle), exchange {n, mean, var} and merge
them (mc.merge); the merged statistics equal a single evaluation over the union.  Also the
max-over-ranks reduction of step times used by bench.py."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2311_17189_gb300 import mc
from paper_2311_17189_gb300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_per_rank, out_dir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = W.ORDER2
    S = O.Solution(c["alpha"], var_is_boson=c["var_is_boson"])
    X = W.matsubara(c["beta"], 3)
    off, n = mc.shard(rank, world, n_per_rank)
    r = S.eval_momenta(W.lattice(c), c["seed"], off, n, X, c["beta"], per_sample=False)
    mine = torch.tensor(np.concatenate([[n], r["mean"].real, r["mean"].imag, r["var"].ravel()]), dtype=torch.float64)
    allv = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(allv, mine)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        nf = len(X)
        stats = []
        for v in allv:
            v = v.numpy()
            stats.append((int(v[0]), v[1:1 + nf] + 1j * v[1 + nf:1 + 2 * nf], v[1 + 2 * nf:].reshape(nf, 2)))
        n_tot, mean, var = mc.merge(stats)
        np.savez(os.path.join(out_dir, "merged.npz"), n=n_tot, mean=mean, var=var, tmax=t.item())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shard_and_merge():
    world, n_per_rank = 2, 20000
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker, args=(world, _free_port(), n_per_rank, d), nprocs=world, join=True)
        got = np.load(os.path.join(d, "merged.npz"))
        import oracle as O
        c = W.ORDER2
        S = O.Solution(c["alpha"], var_is_boson=c["var_is_boson"])
        X = W.matsubara(c["beta"], 3)
        ref = S.eval_momenta(W.lattice(c), c["seed"], 0, world * n_per_rank, X, c["beta"], per_sample=True)
        assert int(got["n"]) == world * n_per_rank
        scale = np.mean(np.abs(ref["values"]), axis=1)
        assert np.all(np.abs(got["mean"] - ref["mean"]) <= 1e-13 * scale)
        assert np.allclose(got["var"], ref["var"], rtol=1e-11, atol=0)
        assert got["tmax"] == 2.0


def test_shard_layout_is_disjoint_and_contiguous_per_step():
    world, n = 4, 1000
    offs = [mc.shard(r, world, n)[0] for r in range(world)]
    assert offs == [0, 1000, 2000, 3000]
    with pytest.raises(ValueError):
        mc.shard(4, 4, n)

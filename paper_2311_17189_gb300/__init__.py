"""Batched evaluation of algorithmic Matsubara integration (AMI, arXiv:2311.17189) on GB300.

    import paper_2311_17189_gb300 as tami
    d = tami.Diagram(alpha, eps=eps)            # AMI construction by residues (host, C++)
    d.upload()                                   # term table to the current CUDA device
    mean, var, _ = d.forward(lattice, seed, 0, n, X, beta)   # Monte Carlo over momenta (CUDA)

Only marshalling lives in Python; the construction is libtami's C++ and every evaluation
step is a libtami CUDA kernel.  `workloads` holds the seeded synthetic inputs.
"""
from . import _lib, mc
from .api import Batch, Diagram, construct_many, debug_set_wait_limit, enumerate_sigma, set_jit, set_table_staging
from . import graph

__all__ = ["Batch", "Diagram", "construct_many", "debug_set_wait_limit", "enumerate_sigma", "graph", "_lib", "mc",
           "set_jit", "set_table_staging"]

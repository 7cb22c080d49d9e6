"""Graph import and labelling (Sec. 2.5) on CPU: libtami's graph labeller reproduces the oracle
enumerator's labels bit for bit when given the same diagram as a graph file, conserves momentum,
and rejects malformed graphs."""
import os

import numpy as np
import pytest

import oracle as O
import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import _lib as L
from paper_2311_17189_gb300 import graph as Gr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("order", [2, 3, 4, 5])
def test_graph_labels_equal_enumerator_labels(order, tmp_path):
    for d in O.enumerate_sigma(order):
        edges = Gr.sigma_graph_from_code(d["code"])
        p = tmp_path / "g.graph"
        Gr.write_graph(edges, p)
        lab = Gr.label_graph(Gr.read_graph(p))
        assert np.array_equal(lab["alpha"], d["alpha"])
        assert np.array_equal(lab["eps"], d["eps"])
        assert lab["loops"] == d["loops"]


def test_second_order_graph_file():
    edges = Gr.read_graph(os.path.join(GOLDEN, "sigma_order2.graph"))
    lab = Gr.label_graph(edges)
    a = lab["alpha"]
    assert a.shape == (3, 3) and lab["loops"] == 1
    assert list(lab["row_line"]) == [0, 1, 2]
    # momentum conservation at the two interaction nodes {0,1} and {2,3} (legs carry k_ext)
    node = {0: 0, 1: 0, 2: 1, 3: 1}
    tot = {0: np.zeros(3, int), 1: np.zeros(3, int)}
    for r, li in enumerate(lab["row_line"]):
        s, t = edges[li, :2]
        tot[node[s]] -= a[r]
        tot[node[t]] += a[r]
    tot[0][2] += 1      # incoming leg enters vertex 0
    tot[1][2] -= 1      # outgoing leg leaves vertex 2
    assert all(np.all(v == 0) for v in tot.values())
    D = Gr.diagram_from_graph(edges, prefactor=-1.0)
    i = D.info()
    assert (i["n_terms"], i["n_fermi_factors"], i["n_g_factors"]) == (4, 8, 4)


def test_graph_errors():
    edges = Gr.read_graph(os.path.join(GOLDEN, "sigma_order2.graph"))
    bad = edges.copy()
    bad[1, 1] = 2                      # vertex 2 gets two incoming fermion lines
    with pytest.raises(L.TamiError) as e:
        Gr.label_graph(bad)
    assert e.value.code == L.TAMI_EINVAL
    with pytest.raises(L.TamiError):
        Gr.label_graph(edges[:, :][[0, 3, 4]])   # no bosonic lines at all

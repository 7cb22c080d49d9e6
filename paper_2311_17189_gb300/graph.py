"""Graph files of self-energy diagrams (Sec. 2.5): plain text, one line per propagator,
four space-separated integers "source target B/F spin" (1 = fermionic, 0 = bosonic).

read_graph / write_graph handle the file; label_graph and Diagram.from_graph call libtami's
labeller (tami_label_graph / tami_construct_from_graph), see include/tami.h for the convention
(one external vertex carrying the two amputated legs, bosonic lines = instantaneous interactions).
"""
import ctypes

import numpy as np

from . import _lib as L
from .api import Diagram


def read_graph(path):
    rows = []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                v = [int(x) for x in line.split()]
                if len(v) != 4:
                    raise ValueError(f"{path}: expected 4 columns, got {line!r}")
                rows.append(v)
    return np.asarray(rows, dtype=np.int32).reshape(-1, 4)


def write_graph(edges, path):
    with open(path, "w") as f:
        for r in np.asarray(edges, dtype=np.int32).reshape(-1, 4):
            f.write(" ".join(str(int(x)) for x in r) + "\n")


def label_graph(edges):
    """Momentum labels of a graph: dict with alpha [N, m+1], eps [N, N], row_line [N], loops."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 4))
    n, nv, lo = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    L.check(L.lib().tami_label_graph(L._np_ptr(e), e.shape[0], 0, None, None, None, ctypes.byref(n),
                                     ctypes.byref(nv), ctypes.byref(lo)))
    a = np.zeros((n.value, nv.value), dtype=np.int8)
    ep = np.zeros((n.value, n.value), dtype=np.int8)
    rl = np.zeros(n.value, dtype=np.int32)
    L.check(L.lib().tami_label_graph(L._np_ptr(e), e.shape[0], n.value, L._np_ptr(a), L._np_ptr(ep),
                                     L._np_ptr(rl), ctypes.byref(n), ctypes.byref(nv), ctypes.byref(lo)))
    return {"alpha": a, "eps": ep, "row_line": rl, "loops": lo.value}


def diagram_from_graph(edges, prefactor=1.0):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 4))
    h = ctypes.c_void_p()
    L.check(L.lib().tami_construct_from_graph(L._np_ptr(e), e.shape[0], float(prefactor), ctypes.byref(h)))
    lab = label_graph(e)
    d = Diagram.__new__(Diagram)
    d._h, d.alpha, d.device, d._ws = h, lab["alpha"], None, None
    d.n_lines, d.n_vars = lab["alpha"].shape
    return d


def sigma_graph_from_code(code):
    """Graph of a Hubbard self-energy diagram given by its canonical contraction code (as returned
    by enumerate_sigma): interaction c has up vertex 2c and down vertex 2c+1, the external vertex
    is 2m; internal up lines (by source), down lines (by source), the two legs, then the bosonic
    lines.  Spin column: 0 up, 1 down."""
    code = list(code)
    m = (len(code) - 1) // 2
    X = 2 * m
    pu = {m: code[0]}
    pd = {}
    for c in range(m):
        pu[c] = code[1 + 2 * c]
        pd[c] = code[2 + 2 * c]
    rows = []
    exit_c = None
    for c in range(m):
        if pu[c] == m:
            exit_c = c
        else:
            rows.append([2 * c, 2 * pu[c], 1, 0])
    for c in range(m):
        rows.append([2 * c + 1, 2 * pd[c] + 1, 1, 1])
    rows.append([X, 2 * pu[m], 1, 0])
    rows.append([2 * exit_c, X, 1, 0])
    for c in range(m):
        rows.append([2 * c, 2 * c + 1, 0, 0])
    return np.asarray(rows, dtype=np.int32)

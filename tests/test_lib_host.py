"""Host-side checks of libtami that need no GPU: the shared library loads and exports every
function include/tami.h declares; its enumerator/labeller and its AMI construction agree with
the oracle's independent ones; malformed input is rejected with the documented codes."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tami.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\**\s+\**(tami_[a-z_0-9]+)\(", src, re.M)))


def test_library_exports_every_declared_function():
    names = declared_functions()
    assert "tami_forward" in names and len(names) >= 10
    lib = ctypes.CDLL(L.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(L.EXPORTS) == names


@pytest.mark.parametrize("order", [2, 3, 4, 5])
def test_enumerator_matches_oracle(order):
    """Same diagrams, same canonical order, same momentum labels, shared energies and loop
    counts as the oracle's separately written enumerator (Sec. 2.5)."""
    lib = T.enumerate_sigma(order)
    orc = O.enumerate_sigma(order)
    assert len(lib) == len(orc)
    for a, b in zip(lib, orc):
        assert a["code"] == b["code"]
        assert np.array_equal(a["alpha"], b["alpha"])
        assert np.array_equal(a["eps"], b["eps"])
        assert a["loops"] == b["loops"]


@pytest.mark.parametrize("order", [2, 3, 4, 5])
def test_construction_counts_match_oracle(order):
    """Term count, factor counts, highest derivative, distinct poles and denominators of the
    library's construction equal the oracle's for every enumerated diagram, in both
    summation orders."""
    for d in T.enumerate_sigma(order):
        for ordr in (None, list(range(order))[::-1]):
            D = T.Diagram(d["alpha"], eps=d["eps"], order=ordr)
            S = O.Solution(d["alpha"], eps=d["eps"], order=ordr)
            a, b = D.info(), S.info()
            assert a["n_terms"] == b["terms"]
            assert a["n_fermi_factors"] == b["fermi_factors"]
            assert a["n_g_factors"] == b["g_factors"]
            for k in ("max_der", "max_g", "unique_poles", "unique_dens"):
                assert a[k] == b[k], k


def test_construction_counts_multipole_and_bosonic_cases():
    cases = [
        ([[1, 0, 1], [0, 1, 0], [1, 1, 0]], None, [1, 0, 0]),
        ([[1, 0], [1, 0], [1, 0], [1, 0], [1, 1]], [[1, 0, 0, 0, 0]] * 4 + [[0, 0, 0, 0, 1]], [0, 1]),
        ([[1, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 1, 1]], [[1, 0, 0, 0], [1, 0, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1]], None),
    ]
    for alpha, eps, boson in cases:
        a = T.Diagram(alpha, eps=eps, var_is_boson=boson).info()
        b = O.Solution(alpha, eps=eps, var_is_boson=boson).info()
        assert (a["n_terms"], a["max_der"], a["unique_poles"], a["unique_dens"]) == \
               (b["terms"], b["max_der"], b["unique_poles"], b["unique_dens"])


EXT_CASES = [
    # (alpha, eps, boson, n_ext): several external frequencies (Sec. 2.3, n_nu > 1)
    ([[1, 1, 0], [1, 0, 1]], None, None, 2),
    ([[1, 0, 0], [1, 1, -1]], None, None, 2),
    ([[1, 1, 0, 0], [1, 0, 1, 0], [1, 0, 0, 1]], None, [0, 1, 0, 0], 3),
    ([[1, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [-1, 1, 1, 1]],
     [[1, 0, 0, 0], [1, 0, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1]], [0, 0, 1, 0], 2),
]


def test_construction_counts_with_several_externals():
    """Library and oracle construct independently; with n_ext external variables they agree on
    the terms, derivative orders and the distinct poles and (energy, external-coefficient)
    denominators, also for the enumerated order-3 and order-4 diagrams with their last internal
    variable held external."""
    cases = list(EXT_CASES)
    for order in (3, 4):
        for d in T.enumerate_sigma(order)[:4]:
            b = [0] * (order + 1)
            b[order - 1] = 1
            cases.append((d["alpha"], d["eps"], b, 2))
    for alpha, eps, boson, n_ext in cases:
        a = T.Diagram(alpha, eps=eps, var_is_boson=boson, n_ext=n_ext).info()
        b = O.Solution(alpha, eps=eps, var_is_boson=boson, n_ext=n_ext).info()
        assert a["n_ext"] == n_ext
        assert (a["n_terms"], a["n_fermi_factors"], a["n_g_factors"], a["max_der"], a["unique_poles"],
                a["unique_dens"]) == (b["terms"], b["fermi_factors"], b["g_factors"], b["max_der"],
                                      b["unique_poles"], b["unique_dens"])


def test_rejects_bad_external_counts():
    for n_ext in (0, 3, 5):
        with pytest.raises(L.TamiError) as e:
            T.Diagram([[1, 1, 0], [1, 0, 1]], n_ext=n_ext)   # n_vars = 3: at most 2 externals
        assert e.value.code == L.TAMI_EINVAL
    assert T.Diagram([[1, 0, 1], [0, 1, 0], [1, 1, 0]], var_is_boson=[1, 0, 0]).info()["n_ext"] == 1


def test_order2_table_shape():
    """The order-2 Hubbard self-energy gives exactly 4 terms with 2 Fermi factors and one
    Green's function each (the two two-leaf sums of Fig. treeflow, multiplied out)."""
    D = T.Diagram([[1, 0, 1], [0, 1, 0], [1, 1, 0]], var_is_boson=[1, 0, 0])
    i = D.info()
    assert (i["n_terms"], i["n_fermi_factors"], i["n_g_factors"], i["max_g"]) == (4, 8, 4, 1)


def test_rejects_malformed_input():
    with pytest.raises(L.TamiError) as e:
        T.Diagram([[2, 0], [1, 1]])
    assert e.value.code == L.TAMI_EINVAL
    with pytest.raises(L.TamiError) as e:
        T.Diagram([[1, 0]])          # a single G decays like 1/z: no residue theorem
    assert e.value.code == L.TAMI_EUNSUPPORTED
    with pytest.raises(L.TamiError) as e:
        T.Diagram([[1, 0, 0], [0, 1, 0], [-1, 1, 1]], order=[0, 0])
    assert e.value.code == L.TAMI_EINVAL
    with pytest.raises(L.TamiError) as e:
        T.Diagram(np.zeros((17, 3), dtype=np.int8))
    assert e.value.code == L.TAMI_EINVAL
    with pytest.raises(L.TamiError):
        T.enumerate_sigma(1)


def test_bench_construct_workload_runs_on_the_host():
    """bench.py --workload construct times the host-side construction without a GPU and prints one
    JSON line: every order-6 diagram constructed, term counts as the library reports them."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "construct", "--steps", "2"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert [d["terms"] for d in line["diagrams"]] == [4, 104, 744, 5136]
    assert line["order6_all"]["diagrams"] == 515 and all(d["ms"] > 0 for d in line["diagrams"])


def test_construct_many_on_host_threads_equals_one_by_one():
    """construct_many builds diagrams on a pool of host threads: the same tables (term counts, flop
    model, generated kernels) in the order of the specs as constructing them one by one; a bad spec
    raises the library's error."""
    specs = [dict(alpha=d["alpha"], eps=d["eps"]) for d in T.enumerate_sigma(5)]
    one = [T.Diagram(**sp) for sp in specs]
    many = T.construct_many(specs, threads=4)
    assert len(many) == len(one)
    for a, b in zip(one, many):
        assert a.info() == b.info()
        assert a.jit_source("fused") == b.jit_source("fused")
    assert T.construct_many([]) == []
    with pytest.raises(L.TamiError):
        T.construct_many(specs[:3] + [dict(alpha=np.zeros((17, 3), dtype=np.int8))], threads=2)

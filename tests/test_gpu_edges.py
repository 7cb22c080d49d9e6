"""Edge cases of the GPU entry points: invalid launches are refused with TAMI_EINVAL before
anything is launched and leave the library usable; an empty energy input launches nothing; the
largest frequency count each kernel accepts evaluates correctly (against the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import _lib as L
from paper_2311_17189_gb300 import workloads as W

import bounds as Bd

pytestmark = pytest.mark.gpu

RTOL = 1e-11


@pytest.fixture(scope="module")
def order2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    c = W.ORDER2
    return T.Diagram(c["alpha"], var_is_boson=c["var_is_boson"]).upload(0), c


def refused(fn):
    with pytest.raises(L.TamiError) as e:
        fn()
    assert e.value.code == L.TAMI_EINVAL, str(e.value)


def test_invalid_launches_are_refused_and_the_library_stays_usable(order2):
    D, c = order2
    lat, beta = W.lattice(c), c["beta"]
    X = W.matsubara(beta, 4)
    g = np.ones(4) + 0.5j
    ref, _, _ = D.forward(lat, c["seed"], 0, 1000, X, beta)
    gref = D.backward(lat, c["seed"], 0, 1000, X, beta, g)
    torch.cuda.synchronize()
    many = W.matsubara(beta, 2049)
    for n, Xb, b in [(0, X, beta), (1000, X[:0], beta), (1000, many, beta), (1000, X, 0.0), (1000, X, -1.0),
                     (1000, X, float("nan")), (1000, X, float("inf"))]:
        refused(lambda: D.forward(lat, c["seed"], 0, n, Xb, b))
    for n, Xb, gb, b in [(0, X, g, beta), (1000, many[:257], np.ones(257) + 0j, beta), (1000, X, g, 0.0),
                         (1000, X, g, float("nan"))]:
        refused(lambda: D.backward(lat, c["seed"], 0, n, Xb, b, gb))
    E = torch.tensor(W.random_energies(10, 3), device="cuda")
    refused(lambda: D.eval_energies(E, X, -2.0))
    empty = D.eval_energies(E[:0].contiguous(), X, beta)
    assert tuple(empty.shape) == (4, 0)
    B = T.Batch([D], [1000], [c["seed"]], len(X))
    refused(lambda: B.launch(lat, X, 0.0))
    U = T.Diagram(c["alpha"], var_is_boson=c["var_is_boson"])          # never uploaded
    refused(lambda: U.forward(lat, c["seed"], 0, 1000, X, beta))
    # the same launches as before the refusals give the same bits
    again, _, _ = D.forward(lat, c["seed"], 0, 1000, X, beta)
    gagain = D.backward(lat, c["seed"], 0, 1000, X, beta, g)
    torch.cuda.synchronize()
    assert torch.equal(again, ref)
    assert torch.equal(gagain["grad_params"], gref["grad_params"])


def test_largest_frequency_counts(order2):
    """2048 frequencies in the forward and 256 in the adjoint (each kernel's limit), ragged sample
    count: per-sample values and per-sample gradients against the oracle."""
    D, c = order2
    S = O.Solution(c["alpha"], var_is_boson=c["var_is_boson"])
    lat, beta = W.lattice(c), c["beta"]
    n = 128 + 3
    X = W.matsubara(beta, 2048)
    _, _, ps = D.forward(lat, c["seed"], 7, n, X, beta, per_sample=True)
    r = S.eval_momenta(lat, c["seed"], 7, n, X, beta, per_sample=True, threads=8)
    assert np.all(np.abs(ps.cpu().numpy() - r["values"]) <= Bd.value_bound(r, lat))
    Xb = W.real_axis(-3.0, 3.0, 256, 0.1)
    g = np.linspace(0.5, 1.5, 256) + 0.25j
    out = D.backward(lat, c["seed"], 7, n, Xb, beta, g, per_sample=True)
    got = out["grads"].cpu().numpy()
    for k, which in enumerate(("mu", "kx", "ky")):
        der, dbd = Bd.oracle_deriv(S, lat, c["seed"], 7, n, Xb, beta, which)
        ref = np.real(np.conj(g)[:, None] * der).sum(axis=0)
        assert np.all(np.abs(got[:, k] - ref) <= (np.abs(g)[:, None] * dbd).sum(axis=0)), which


def test_nvtx_ranges_change_nothing(order2, monkeypatch):
    """TAMI_NVTX=1 wraps the library calls in NVTX ranges for timeline profilers; the results are
    the same bits."""
    D, c = order2
    lat, beta = W.lattice(c), c["beta"]
    X = W.matsubara(beta, 3)
    ref, _, _ = D.forward(lat, c["seed"], 0, 777, X, beta)
    monkeypatch.setenv("TAMI_NVTX", "1")
    got, _, _ = D.forward(lat, c["seed"], 0, 777, X, beta)
    g = D.backward(lat, c["seed"], 0, 777, X, beta, np.ones(3) + 0j)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    assert torch.all(torch.isfinite(g["grad_params"]))

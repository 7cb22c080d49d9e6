"""Large term tables on the GPU: the pole-DAG program streamed through shared memory in chunks
(tables whose program does not fit beside the tiles), order-6 self-energy diagrams (the paper's
scaling study runs to orders 6 and 9, Sec. 6.2) against the oracle, diagrams built from graph
files (Sec. 2.5) against the oracle, and the staging wait running out on a valid copy.

Bounds as in test_gpu_forward.py / test_gpu_adjoint.py (tests/bounds.py): 1e-11 of the oracle's
rounding envelope plus the input part for the two sides' cos/sin.  Streamed and resident staging
run the same arithmetic, so they are compared bit for bit.
"""
import functools
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import graph as Gr
from paper_2311_17189_gb300 import workloads as W

import bounds as B

pytestmark = pytest.mark.gpu

RTOL = B.RTOL
LAT = (1.0, -0.2, 0.1, np.pi / 2, np.pi / 3)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.fixture
def modes():
    """Staging, specialisation and wait limit for one test, restored afterwards."""
    yield
    T.set_table_staging("auto", 512)
    T.set_jit("auto")
    T.debug_set_wait_limit(-1)


def enumerated(order, code):
    return next(d for d in O.enumerate_sigma(order) if d["code"] == tuple(code))


def pair(d, prefactor=1.0):
    D = T.Diagram(d["alpha"], eps=d["eps"], prefactor=prefactor).upload(0)
    S = O.Solution(d["alpha"], eps=d["eps"], prefactor=prefactor)
    return D, S


def optin():
    return torch.cuda.get_device_properties(0).shared_memory_per_block_optin


# ---------------------------------------------------------------------------- streamed program
@pytest.mark.parametrize("chunk", [16, 18, 512, 4096])
def test_streamed_program_gives_resident_bits(modes, chunk):
    """The forward pole-DAG program streamed through the two-buffer ring (chunk ops per buffer:
    16 and 18 cross hundreds of chunk boundaries and end on a ragged chunk, 4096 holds the whole
    program in one) gives the resident program's bits: per-sample values, saved rows, mean and
    variance, on the order-4 bench table and the largest order-5 table, with a ragged last tile;
    and energy input on the order-5 table."""
    T.set_jit("never")
    n = 3 * 128 + 37
    for order, code in ((4, W.ORDER4["code"]), (5, W.ORDER5["code"])):
        D, _ = pair(enumerated(order, code))
        X = W.matsubara(5.0, 3)
        T.set_table_staging("auto")
        sv0 = D.saved_buffer(n)
        m0, v0, p0 = D.forward(LAT, 7, 11, n, X, 5.0, per_sample=True, save=sv0)
        E = torch.as_tensor(W.random_energies(300, D.n_lines, a=4.0, seed=3), device="cuda")
        e0 = D.eval_energies(E, X, 5.0)
        T.set_table_staging("streamed", chunk)
        sv1 = D.saved_buffer(n)
        m1, v1, p1 = D.forward(LAT, 7, 11, n, X, 5.0, per_sample=True, save=sv1)
        e1 = D.eval_energies(E, X, 5.0)
        torch.cuda.synchronize()
        assert torch.equal(p0, p1) and torch.equal(sv0, sv1), (order, chunk)
        assert torch.equal(m0, m1) and torch.equal(v0, v1), (order, chunk)
        assert torch.equal(e0, e1), (order, chunk)


def test_streamed_batch_gives_resident_bits(modes):
    """A persistent batch plan (generic kernel, orders 2-4 mixed) with every program streamed in
    chunks of 16 ops gives the resident plan's bits."""
    T.set_jit("never")
    lib = []
    for m in (2, 3, 4):
        for d in O.enumerate_sigma(m)[:3]:
            lib.append(T.Diagram(d["alpha"], eps=d["eps"]).upload(0))
    counts = [1000 + 517 * k for k in range(len(lib))]
    seeds = [40 + k for k in range(len(lib))]
    X = W.matsubara(5.0, 4)
    T.set_table_staging("auto")
    b0 = T.Batch(lib, counts, seeds, len(X), chunk_tiles=2)
    m0, v0 = b0.launch(LAT, X, 5.0)
    T.set_table_staging("streamed", 16)
    b1 = T.Batch(lib, counts, seeds, len(X), chunk_tiles=2)
    m1, v1 = b1.launch(LAT, X, 5.0)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(m0)).all()
    assert torch.equal(m0, m1) and torch.equal(v0, v1)


# ---------------------------------------------------------------------------- order 6
@functools.lru_cache(maxsize=1)
def order6_cases():
    """Order-6 diagrams: the largest flat table, the table with the largest generic-forward shared
    memory, the first table whose terms need second Fermi derivatives (third in the adjoint), and
    two others, chosen from the library's own table sizes."""
    ds = O.enumerate_sigma(6)
    infos = [T.Diagram(d["alpha"], eps=d["eps"]).info() for d in ds]
    terms = [i["n_terms"] for i in infos]
    smem = [i["table_bytes"] + 8 * 128 * (i["n_cplx_dens"] + i["n_groups_freq"]) for i in infos]
    second = next(k for k, i in enumerate(infos) if i["max_der"] >= 2)
    picks = [int(np.argmax(terms)), int(np.argmax(smem)), second, len(ds) // 3, 2 * len(ds) // 3]
    return ds, infos, list(dict.fromkeys(picks))


def test_order6_enumeration_and_tables():
    """515 order-6 diagrams (the two enumerators agree), every one constructs, the largest flat
    table has 5136 terms, and the deepest Fermi derivative any of them needs is the second (the
    oracle's construction agrees on it)."""
    ds, infos, picks = order6_cases()
    assert len(ds) == 515 == len(T.enumerate_sigma(6))
    assert max(i["n_terms"] for i in infos) == 5136
    assert max(i["max_der"] for i in infos) == 2
    second = next(k for k, i in enumerate(infos) if i["max_der"] >= 2)
    assert second in picks
    d = ds[second]
    assert O.Solution(d["alpha"], eps=d["eps"]).info()["max_der"] == 2
    for i, d in enumerate(ds[::37]):
        S = O.Solution(d["alpha"], eps=d["eps"])
        assert S.info()["terms"] == infos[37 * i]["n_terms"]


def test_order6_forward_and_adjoint_against_oracle(modes):
    """Order-6 tables per sample against the oracle: the forward (generic kernel, program resident
    or streamed as it fits) and the fused forward + adjoint -- values, dSigma/dX and the contracted
    gradients.  The largest tables exceed the generic adjoint's per-thread capacities, so the
    default mode specialises them at any size; a table the generic adjoint holds (the one with
    second Fermi derivatives) is checked through both kernel families."""
    ds, infos, picks = order6_cases()
    X = W.matsubara(5.0, 2)
    g = np.array([1.0 + 0.5j, -0.25 + 1.0j])
    n, seed, off = 3 * 128 + 37, 23, 1000
    for i in picks:
        d = ds[i]
        pref = (-1.0) ** 6 * (-1.0) ** d["loops"]
        D, S = pair(d, pref)
        m, v, ps = D.forward(LAT, seed, off, n, X, 5.0, per_sample=True)
        runs = [D.forward_backward(LAT, seed, off, n, X, 5.0, g, per_sample=True)]
        torch.cuda.synchronize()
        if i == int(np.argmax([f["n_terms"] for f in infos])):
            assert D.jit_status()["last_used"], i      # the fused pass ran the specialised kernel
        if not D.jit_status()["last_used"]:
            T.set_jit("always")
            runs.append(D.forward_backward(LAT, seed, off, n, X, 5.0, g, per_sample=True))
            torch.cuda.synchronize()
            assert D.jit_status()["last_used"], i
            T.set_jit("auto")
        ref = S.eval_momenta(LAT, seed, off, n, X, 5.0, per_sample=True, threads=16)
        vb = B.value_bound(ref, LAT)
        assert np.all(np.abs(m.cpu().numpy() - ref["mean"]) <= RTOL * B.mean_scale(ref, LAT)), i
        dref, dbd = B.oracle_deriv(S, LAT, seed, off, n, X, 5.0, "omega", threads=16)
        gders = [B.oracle_deriv(S, LAT, seed, off, n, X, 5.0, w, threads=16) for w in ("mu", "kx", "ky")]
        for got in [ps] + [fb["values"] for fb in runs]:
            err = np.abs(got.cpu().numpy() - ref["values"])
            assert np.all(err <= vb), (i, np.max(err / vb))
        for fb in runs:
            assert np.all(np.abs(fb["dX"].cpu().numpy() - dref) <= dbd), i
            grads = fb["grads"].cpu().numpy()
            for k, (der, gbd) in enumerate(gders):
                gref = np.real(np.conj(g)[:, None] * der).sum(axis=0)
                assert np.all(np.abs(grads[:, k] - gref) <= (np.abs(g)[:, None] * gbd).sum(axis=0)), (i, k)


def test_order6_program_streamed_where_it_does_not_fit(modes):
    """The order-6 table with the largest generic-forward footprint at a frequency count where the
    resident program no longer fits beside the tiles: the default staging streams it, and the
    per-sample values still meet the oracle (energy input, so only the rounding bound applies)."""
    ds, infos, _ = order6_cases()
    i = int(np.argmax([x["table_bytes"] + 8 * 128 * (x["n_cplx_dens"] + x["n_groups_freq"]) for x in infos]))
    D, S = pair(ds[i])
    h = D.info()
    # the blob ends with the two programs (8 bytes per op, each padded to 16) and 16 spare bytes;
    # resident: [0, off_opsb) + per-frequency rows + tiles; streamed: [0, off_ops) + the ring instead
    prog = (8 * h["n_dag_ops"] + 15) // 16 * 16
    off_opsb = h["table_bytes"] - 16 - prog
    tiles = 8 * 128 * (h["n_cplx_dens"] + h["n_groups_freq"] + 4)
    per_f = 8 * (2 + 2 * h["n_cplx_dens"])
    resident0 = off_opsb + tiles
    n_f = max(1, (optin() - resident0) // per_f + 1)
    streamed = resident0 - prog + 2 * 8 * 512 + per_f * n_f
    if streamed > optin():
        pytest.skip("no frequency count separates the two stagings for this table")
    T.set_jit("never")
    X = W.matsubara(5.0, int(n_f))
    E = W.random_energies(40, D.n_lines, a=3.0, seed=8)
    E = E[:, np.asarray(ds[i]["eps"]).argmax(1)]
    got = D.eval_energies(torch.as_tensor(E, device="cuda"), X, 5.0).cpu().numpy()
    ref, _, env = S.eval_energies(E, X, 5.0, threads=16)
    assert np.all(np.abs(got - ref) <= RTOL * env)


# ---------------------------------------------------------------------------- graph files
def test_graph_file_diagrams_against_oracle(tmp_path):
    """Diagrams built from graph files (Sec. 2.5: read, label, construct): the second-order
    self-energy of tests/golden/sigma_order2.graph and an order-4 diagram written to a file from
    its contraction code, each evaluated on the GPU per sample against the oracle built from the
    labels the file gives."""
    e2 = Gr.read_graph(os.path.join(GOLDEN, "sigma_order2.graph"))
    d4 = enumerated(4, W.ORDER4["code"])
    p = tmp_path / "order4.graph"
    Gr.write_graph(Gr.sigma_graph_from_code(d4["code"]), p)
    e4 = Gr.read_graph(p)
    X = W.matsubara(8.0, 4)
    lat = W.lattice(W.ORDER4)
    for edges in (e2, e4):
        lab = Gr.label_graph(edges)
        D = Gr.diagram_from_graph(edges, prefactor=-1.0).upload(0)
        S = O.Solution(lab["alpha"], eps=lab["eps"], prefactor=-1.0)
        assert D.info()["n_terms"] == S.info()["terms"]
        n = 3 * 128 + 5
        _, _, ps = D.forward(lat, 5, 0, n, X, 8.0, per_sample=True)
        ref = S.eval_momenta(lat, 5, 0, n, X, 8.0, per_sample=True, threads=8)
        assert np.all(np.abs(ps.cpu().numpy() - ref["values"]) <= B.value_bound(ref, lat))


# ---------------------------------------------------------------------------- bounded waits
def test_staging_wait_running_out_is_reported(modes):
    """With the first stage of every staging wait bounded to zero polls, each wait 'runs out' on a
    valid copy: the status word is set, so the reduced outputs are NaN, while the copy is still
    waited for (second, bounded stage) and the per-sample values keep their bits.  The forward
    (program resident and streamed), the fused forward + adjoint and a batch plan; with the
    default limit restored the next calls give the earlier bits.  No fault and no unbounded wait
    is involved."""
    T.set_jit("never")
    c = W.ORDER2
    D = T.Diagram(c["alpha"], var_is_boson=c["var_is_boson"]).upload(0)
    lat, beta, n = W.lattice(c), c["beta"], 1000
    X = W.matsubara(beta, 2)
    g = np.array([1.0 + 0.5j, -0.25 + 1.0j])
    m0, v0, p0 = D.forward(lat, c["seed"], 0, n, X, beta, per_sample=True)
    f0 = D.forward_backward(lat, c["seed"], 0, n, X, beta, g, per_sample=True)
    b0 = T.Batch([D], [n], [c["seed"]], len(X), chunk_tiles=2)
    bm0, _ = b0.launch(lat, X, beta)
    torch.cuda.synchronize()
    T.debug_set_wait_limit(0)
    for mode in ("auto", "streamed"):
        T.set_table_staging(mode, 16)
        m1, v1, p1 = D.forward(lat, c["seed"], 0, n, X, beta, per_sample=True)
        torch.cuda.synchronize()
        assert torch.isnan(torch.view_as_real(m1)).all() and torch.isnan(v1).all(), mode
        assert torch.equal(p1, p0), mode
    T.set_table_staging("auto", 512)
    f1 = D.forward_backward(lat, c["seed"], 0, n, X, beta, g, per_sample=True)
    b1 = T.Batch([D], [n], [c["seed"]], len(X), chunk_tiles=2)
    bm1, _ = b1.launch(lat, X, beta)
    torch.cuda.synchronize()
    assert torch.isnan(torch.view_as_real(f1["mean"])).all() and torch.isnan(f1["grad_params"]).all()
    assert torch.equal(f1["values"], f0["values"]) and torch.equal(f1["grads"], f0["grads"])
    assert torch.isnan(torch.view_as_real(bm1)).all()
    T.debug_set_wait_limit(-1)
    m2, v2, p2 = D.forward(lat, c["seed"], 0, n, X, beta, per_sample=True)
    f2 = D.forward_backward(lat, c["seed"], 0, n, X, beta, g, per_sample=True)
    b2 = T.Batch([D], [n], [c["seed"]], len(X), chunk_tiles=2)
    bm2, _ = b2.launch(lat, X, beta)
    torch.cuda.synchronize()
    assert torch.equal(m2, m0) and torch.equal(v2, v0) and torch.equal(p2, p0)
    assert torch.equal(f2["mean"], f0["mean"]) and torch.equal(f2["grad_params"], f0["grad_params"])
    assert torch.equal(bm2, bm0)


@pytest.mark.parametrize("beta", [2.0, 20.0])
def test_order6_workload_full_size_sampled(beta):
    """The order-6 workload at its full size (the 5136-term table, 2^24 samples, one frequency
    i pi/beta; the specialised kernels at this size): per-sample values at 200 random samples
    against the oracle one by one, the mean against the mean of all per-sample outputs, the fused
    forward + adjoint's per-sample dSigma/dX and contracted gradients at 30 random samples against
    the oracle's dual numbers, and a second full launch equal bit for bit."""
    c = W.ORDER6
    d = enumerated(6, c["code"])
    D, S = pair(d)
    assert D.info()["n_terms"] == S.info()["terms"] == 5136
    X = W.matsubara(beta, c["n_freq"])
    n, lat = c["n_samples"], W.lattice(c)
    mean, var, ps = D.forward(lat, c["seed"], 0, n, X, beta, per_sample=True)
    torch.cuda.synchronize()
    assert D.jit_status()["last_used"]
    rng = np.random.default_rng(int(beta) + 6)
    idx = np.sort(rng.choice(n, 200, replace=False))
    got = ps[:, torch.as_tensor(idx, device="cuda")].cpu().numpy()
    plain = []
    for k, i in enumerate(idx):
        r = S.eval_momenta(lat, c["seed"], int(i), 1, X, beta, per_sample=True)
        err = np.abs(got[:, k] - r["values"][:, 0])
        assert np.all(err <= B.value_bound(r, lat)[:, 0]), (i, err, r["envelope"][:, 0])
        plain.append(np.mean(err <= RTOL * np.abs(r["values"][:, 0])))
    print(f"order-6 workload, beta {beta}: {np.mean(plain):.4f} of sampled values within plain relative 1e-11")
    ps_mean = ps.mean(dim=1).cpu().numpy()
    scale = ps.abs().mean(dim=1).cpu().numpy()
    assert np.all(np.abs(mean.cpu().numpy() - ps_mean) <= 1e-12 * scale)
    del ps
    g = np.array([1.0 + 0.5j])
    fb = D.forward_backward(lat, c["seed"], 0, n, X, beta, g, per_sample=True)
    again = D.forward_backward(lat, c["seed"], 0, n, X, beta, g)
    torch.cuda.synchronize()
    assert torch.equal(fb["grad_params"], again["grad_params"]) and torch.equal(fb["mean"], again["mean"])
    ti = torch.as_tensor(idx[:30], device="cuda")
    dX = fb["dX"][:, ti].cpu().numpy()
    grads = fb["grads"][ti].cpu().numpy()
    for k, i in enumerate(idx[:30]):
        dref, dbd = B.oracle_deriv(S, lat, c["seed"], int(i), 1, X, beta, "omega", threads=1)
        assert np.all(np.abs(dX[:, k] - dref[:, 0]) <= dbd[:, 0]), i
        for j, which in enumerate(("mu", "kx", "ky")):
            der, dbd = B.oracle_deriv(S, lat, c["seed"], int(i), 1, X, beta, which, threads=1)
            ref = np.real(np.conj(g) * der[:, 0]).sum()
            assert abs(grads[k, j] - ref) <= (np.abs(g) * dbd[:, 0]).sum(), (i, which)

"""GPU tests of the persistent multi-diagram launch (tami_batch_*): every diagram's mean and
variance against the CPU oracle, against separate tami_forward launches on the same samples,
determinism of a plan, the autotuner and its cache, and the full all-orders workload; plans whose
diagrams run their specialised forward kernels (all of them, or the large ones beside the
persistent kernel), the parameters such a captured plan reads at each launch, and the kernels a
plan keeps after its diagrams are gone."""
import gc
import os

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


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def mixed_batch():
    """Diagrams of orders 2..5 with uneven sample counts (a single sample, ragged tails)."""
    picks = [(2, 0), (3, 1), (4, 2), (4, 7), (5, 3), (5, 40)]
    counts = [1, 3 * 128 + 37, 5000, 129, 2000, 700]
    ds = [O.enumerate_sigma(m)[i] for m, i in picks]
    lib = [T.Diagram(d["alpha"], eps=d["eps"], prefactor=(-1.0) ** m * (-1.0) ** d["loops"])
           for d, (m, _) in zip(ds, picks)]
    orc = [O.Solution(d["alpha"], eps=d["eps"], prefactor=(-1.0) ** m * (-1.0) ** d["loops"])
           for d, (m, _) in zip(ds, picks)]
    seeds = [W.SEED + k for k in range(len(ds))]
    return lib, orc, counts, seeds


LAT = (1.0, -0.2, 0.1, np.pi / 2, np.pi / 3)
BETA = 5.0


@pytest.fixture
def jit():
    """set_jit for one test, restored to the default afterwards."""
    yield T.set_jit
    T.set_jit("auto")


def check_against_oracle(mean, var, orc, counts, seeds, X):
    mean, var = mean.cpu().numpy(), var.cpu().numpy()
    for d, (S, n, sd) in enumerate(zip(orc, counts, seeds)):
        ref = S.eval_momenta(LAT, sd, 0, n, X, BETA, per_sample=True, threads=8)
        scale = Bd.mean_scale(ref, LAT)
        assert np.all(np.abs(mean[d] - ref["mean"]) <= RTOL * scale), d
        dev = ref["values"] - ref["mean"][:, None]
        for part, k in ((np.real, 0), (np.imag, 1)):
            tol = 2.0 / max(n - 1, 1) * np.sum(np.abs(part(dev)) * Bd.value_bound(ref, LAT), axis=1) \
                + 1e-10 * ref["var"][:, k]
            assert np.all(np.abs(var[d][:, k] - ref["var"][:, k]) <= tol), d


@pytest.mark.parametrize("chunk", [1, 3])
def test_batch_against_oracle(chunk):
    lib, orc, counts, seeds = mixed_batch()
    X = W.matsubara(BETA, 5)
    B = T.Batch(lib, counts, seeds, len(X), chunk_tiles=chunk)
    assert B.info()["chunk_tiles"] == chunk and B.info()["specialised"] == 0
    mean, var = B.launch(LAT, X, BETA)
    torch.cuda.synchronize()
    check_against_oracle(mean, var, orc, counts, seeds, X)


def test_specialised_batch_against_oracle(jit):
    """Mode "always": every diagram runs its own generated forward kernel in the plan's graph (no
    work items); means and variances meet the oracle bar as the persistent kernel's do."""
    jit("always")
    lib, orc, counts, seeds = mixed_batch()
    X = W.matsubara(BETA, 5)
    B = T.Batch(lib, counts, seeds, len(X))
    info = B.info()
    assert info["specialised"] == len(lib) and info["items"] == 0 and info["grid"] == 0
    mean, var = B.launch(LAT, X, BETA)
    torch.cuda.synchronize()
    check_against_oracle(mean, var, orc, counts, seeds, X)


def single_calls(lib, counts, seeds, lat, X, beta):
    """Each diagram's tami_forward over its batch samples (the current mode picks the kernel):
    means, variances and the mean per-sample magnitude."""
    out = []
    for d, D in enumerate(lib):
        D.upload(0)
        m, v, ps = D.forward(lat, seeds[d], 0, counts[d], X, beta, per_sample=True)
        out.append((m, v, ps.abs().mean(dim=1)))
    return out


def same_code_close(mean, var, ref, rel=1e-12):
    """Batch results against single calls running the same kernel code: they differ only in how
    the partial sums are grouped."""
    for d, (m, v, scale) in enumerate(ref):
        assert torch.all((mean[d] - m).abs() <= rel * scale), d
        assert torch.allclose(var[d], v, rtol=1e-10, atol=0), d


def test_specialised_batch_reads_each_launchs_parameters(jit):
    """The specialised kernels are captured once; a later launch with another lattice, beta and
    frequencies (same count) must use them, as single calls with those inputs do."""
    lib, orc, counts, seeds = mixed_batch()
    X1, X2 = W.matsubara(BETA, 6), W.real_axis(-1.5, 2.5, 6, 0.2)
    lat2, beta2 = (0.8, 0.25, -0.3, 0.4, -1.1), 3.0
    jit("always")
    B = T.Batch(lib, counts, seeds, 6)
    assert B.info()["specialised"] == len(lib)
    r1 = single_calls(lib, counts, seeds, LAT, X1, BETA)
    r2 = single_calls(lib, counts, seeds, lat2, X2, beta2)
    for _ in range(2):
        m1, v1 = B.launch(LAT, X1, BETA)
        m2, v2 = B.launch(lat2, X2, beta2)
        torch.cuda.synchronize()
        same_code_close(m1, v1, r1)
        same_code_close(m2, v2, r2)
        assert not torch.allclose(m1, m2)


def test_auto_mixes_specialised_and_persistent_diagrams(jit):
    """Mode "auto": the diagram with 2^20 samples takes its specialised kernel, the others stay
    work items of the persistent kernel in the same graph.  Results repeat bit for bit; the
    persistent kernel's diagrams give the bits of a plan without specialised kernels, the
    specialised one agrees with its single specialised call."""
    lib, orc, counts, seeds = mixed_batch()
    counts = [1 << 20] + counts[1:]
    X = W.matsubara(BETA, 8)
    jit("auto")
    B = T.Batch(lib, counts, seeds, len(X), chunk_tiles=2)
    info = B.info()
    assert info["specialised_diagrams"] == [0] and info["items"] >= 1
    m1, v1 = B.launch(LAT, X, BETA)
    m2, v2 = B.launch(LAT, X, BETA)
    jit("never")
    G = T.Batch(lib, counts, seeds, len(X), chunk_tiles=2)
    assert G.info()["specialised"] == 0
    g, gv = G.launch(LAT, X, BETA)
    torch.cuda.synchronize()
    assert torch.equal(m1, m2) and torch.equal(v1, v2)
    assert torch.equal(m1[1:], g[1:]) and torch.equal(v1[1:], gv[1:])
    jit("always")
    ref = single_calls(lib[:1], counts[:1], seeds[:1], LAT, X, BETA)
    assert lib[0].jit_status()["last_used"]
    same_code_close(m1[:1], v1[:1], ref)


def test_plan_keeps_its_kernels_after_the_diagrams_are_destroyed(jit):
    jit("always")
    lib, orc, counts, seeds = mixed_batch()
    X = W.matsubara(BETA, 3)
    B = T.Batch(lib, counts, seeds, len(X))
    m1, v1 = B.launch(LAT, X, BETA)
    torch.cuda.synchronize()
    B.diagrams = []
    del lib
    gc.collect()
    m2, v2 = B.launch(LAT, X, BETA)
    torch.cuda.synchronize()
    assert torch.equal(m1, m2) and torch.equal(v1, v2)


def test_specialised_limits_in_batches(jit):
    """More frequencies than the specialised kernels' per-thread sums hold (256): "always" refuses
    the plan, "auto" keeps every diagram on the persistent kernel."""
    lib, orc, counts, seeds = mixed_batch()
    jit("always")
    with pytest.raises(L.TamiError) as e:
        T.Batch(lib[:1], [1 << 20], seeds[:1], 300, chunk_tiles=4)
    assert e.value.code == L.TAMI_EUNSUPPORTED
    jit("auto")
    B = T.Batch(lib[:1], [1 << 20], seeds[:1], 300, chunk_tiles=4)
    assert B.info()["specialised"] == 0 and B.info()["items"] >= 1


def test_batch_matches_single_launches_and_is_deterministic():
    lib, orc, counts, seeds = mixed_batch()
    X = W.real_axis(-2.0, 2.0, 40, 0.1)
    for D in lib:
        D.upload(0)
    B = T.Batch(lib, counts, seeds, len(X), chunk_tiles=2)
    m1, v1 = B.launch(LAT, X, BETA)
    m2, v2 = B.launch(LAT, X, BETA)
    torch.cuda.synchronize()
    assert torch.equal(m1, m2) and torch.equal(v1, v2)
    for d, D in enumerate(lib):
        m, v, ps = D.forward(LAT, seeds[d], 0, counts[d], X, BETA, per_sample=True)
        scale = ps.abs().mean(dim=1)
        assert torch.all((m1[d] - m).abs() <= 1e-13 * scale)


def test_autotune_and_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("TAMI_TUNE_CACHE", str(tmp_path / "tune.txt"))
    monkeypatch.setenv("TAMI_TUNE_LOG", str(tmp_path / "tune.log"))
    lib, orc, counts, seeds = mixed_batch()
    counts = [c * 40 for c in counts]
    X = W.matsubara(BETA, 8)
    B1 = T.Batch(lib, counts, seeds, len(X), chunk_tiles=0)
    i1 = B1.info()
    assert i1["chunk_tiles"] >= 1 and i1["items"] >= 1 and i1["grid"] >= 1
    text = (tmp_path / "tune.txt").read_text()
    assert len(text.strip().splitlines()) == 1
    # the sweep record: every timed candidate, the chosen (chunk, grid) among them
    log = (tmp_path / "tune.log").read_text().strip().splitlines()
    cands = [dict(kv.split("=") for kv in line.split()[1:]) for line in log]
    assert len(cands) >= 2 and all(float(c["ms"]) > 0 for c in cands)
    assert any(int(c["chunk"]) == i1["chunk_tiles"] and int(c["grid"]) == i1["grid"] for c in cands)
    B2 = T.Batch(lib, counts, seeds, len(X), chunk_tiles=0)          # cache hit: no new line
    assert B2.info()["chunk_tiles"] == i1["chunk_tiles"]
    assert (tmp_path / "tune.txt").read_text() == text
    assert len((tmp_path / "tune.log").read_text().strip().splitlines()) == len(log)   # nothing timed
    m1, _ = B1.launch(LAT, X, BETA)
    m2, _ = B2.launch(LAT, X, BETA)
    assert torch.equal(m1, m2)


def test_batch_rejects_bad_arguments():
    lib, orc, counts, seeds = mixed_batch()
    with pytest.raises(L.TamiError):
        T.Batch(lib, counts, seeds, 0)
    with pytest.raises(L.TamiError):
        T.Batch(lib, [0] + counts[1:], seeds, 4)


def test_poisoned_queue_entry_is_refused_without_a_fault():
    """Failure detection of the persistent launch, injected on the host: a queue entry naming a
    diagram or tiles outside the plan is skipped by the kernel (none of the accesses it describes
    is made), the status word marks the launch and every mean and variance comes back NaN; with
    the entry restored, the same plan gives the original results bit for bit."""
    lib, orc, counts, seeds = mixed_batch()
    X = W.matsubara(BETA, 4)
    for D in lib:
        D.upload(0)
    B = T.Batch(lib, counts, seeds, len(X), chunk_tiles=2)
    m0, v0 = B.launch(LAT, X, BETA)
    torch.cuda.synchronize()
    item = B.info()["items"] // 2
    tiles0 = (counts[0] + 127) // 128
    for bad in [(len(lib), 0, 1), (-1, 0, 1), (0, 0, tiles0 + 1), (0, 0, 1 << 40), (0, 1, 1), (0, -3, 1)]:
        prev = B.debug_set_item(item, *bad)
        m, v = B.launch(LAT, X, BETA)
        torch.cuda.synchronize()
        assert torch.all(torch.isnan(m.real)) and torch.all(torch.isnan(v)), bad
        assert B.debug_set_item(item, *prev) == bad
    m1, v1 = B.launch(LAT, X, BETA)
    torch.cuda.synchronize()
    assert torch.equal(m1, m0) and torch.equal(v1, v0)


@pytest.mark.parametrize("mode", ["never", "auto"])
def test_all_orders_workload_full_size(mode, jit):
    """Every Hubbard self-energy diagram of orders 2..5 (85 diagrams), diagram d with
    2^(20 + d mod 4) samples and seed 20231128 + d, 32 Matsubara frequencies, beta = 5, in one
    graph launch: the persistent kernel over every diagram ("never"), or every diagram's
    specialised forward kernel ("auto": all have >= 2^20 samples).  Each diagram's mean against a
    separate tami_forward launch over the same samples running the same code (the generic kernel,
    whose tile code the persistent kernel shares, or the diagram's specialised kernel), so the two
    differ only in how partial sums are grouped.  The two kernel families differ by more than that
    (their multiply-adds are contracted differently, and the terms cancel), so each meets the
    oracle bar in its own small-size tests instead."""
    c = W.ALL_ORDERS
    diags, lib = [], []
    for m in c["orders"]:
        for d in T.enumerate_sigma(m):
            diags.append((m, d))
            lib.append(T.Diagram(d["alpha"], eps=d["eps"], prefactor=(-1.0) ** m * (-1.0) ** d["loops"]))
    n_d = len(lib)
    largest = int(np.argmax([D.info()["n_terms"] for D in lib]))
    sampled = sorted({0, 1, 14, largest})      # orders 2, 3, 4 and the largest order-5 table
    assert n_d == 85
    counts = [W.all_orders_samples(d) for d in range(n_d)]
    seeds = [c["seed"] + d for d in range(n_d)]
    X = W.matsubara(c["beta"], c["n_freq"])
    lat = W.lattice(c)
    jit(mode)
    B = T.Batch(lib, counts, seeds, len(X), chunk_tiles=16)
    assert B.info()["specialised"] == (n_d if mode == "auto" else 0)
    mean, var = B.launch(lat, X, c["beta"])
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(mean)).all()
    jit("always" if mode == "auto" else "never")
    rng = np.random.default_rng(11)
    for d, D in enumerate(lib):
        D.upload(0)
        m, v, ps = D.forward(lat, seeds[d], 0, counts[d], X, c["beta"], per_sample=d in sampled)
        assert D.jit_status()["last_used"] == (mode == "auto")
        rms = torch.sqrt(v.sum(dim=1) + m.abs() ** 2)
        assert torch.all((mean[d] - m).abs() <= 1e-12 * rms), d
        assert torch.allclose(var[d], v, rtol=1e-9, atol=0)
        if d in sampled:
            # per-sample values of the same kernel at 40 random samples against the oracle
            order, dd = diags[d]
            od = next(x for x in O.enumerate_sigma(order) if x["code"] == dd["code"])
            S = O.Solution(od["alpha"], eps=od["eps"], prefactor=(-1.0) ** order * (-1.0) ** od["loops"])
            idx = np.sort(rng.choice(counts[d], 40, replace=False))
            vals = ps[:, torch.as_tensor(idx, device=ps.device)].cpu().numpy()
            for k, i in enumerate(idx):
                r = S.eval_momenta(lat, seeds[d], int(i), 1, X, c["beta"], per_sample=True)
                assert np.all(np.abs(vals[:, k] - r["values"][:, 0]) <= Bd.value_bound(r, lat)[:, 0]), (d, i)
            del ps

"""GPU parity of the specialised fused forward + adjoint kernels (generated per table and compiled
with NVRTC, tami_jit.cpp) against the CPU oracle, and their agreement with the generic kernel.

Per-sample bounds as in test_gpu_forward.py / test_gpu_adjoint.py: 1e-11 of the oracle's rounding
envelope for values, of its derivative envelope for dSigma/dX and the contracted gradients, plus
the input part for the two sides' cos/sin (tests/bounds.py).
Reduced means and variances of the two kernel families agree to the rounding of their sums; their
adjoints round differently per sample (the specialised ones sum shared partial sums' adjoints
once), so reduced derivatives agree to the mean per-sample difference, which stays within the
envelope bound.
"""
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


@pytest.fixture(autouse=True)
def _restore_mode():
    yield
    T.set_jit("auto")


def upstream(n_f, seed=3):
    r = np.random.default_rng(seed)
    return r.normal(size=n_f) + 1j * r.normal(size=n_f)


def order4_bench():
    c = W.ORDER4
    return next(x for x in O.enumerate_sigma(4) if x["code"] == c["code"])


CASES = [
    # name, diagram, lattice, beta, X
    ("order2_bosonic_transfer", dict(alpha=W.ORDER2["alpha"], eps=None, boson=W.ORDER2["var_is_boson"]),
     W.lattice(W.ORDER2), 5.0, W.matsubara(5.0, 3)),
    ("order3_real_axis", (3, 0), (1.0, 0.0, 0.0, np.pi / 2, np.pi / 2), 10.0, W.real_axis(-4.0, 4.0, 7, 0.05)),
    ("order4_bench", "bench", W.lattice(W.ORDER4), 8.0, W.matsubara(8.0, 16)),
    ("order5_real_axis", (5, 7), (1.0, -0.2, 0.1, np.pi / 2, np.pi / 3), 5.0, W.real_axis(-2.0, 2.0, 3, 0.1)),
    ("quadruple_pole", dict(alpha=[[1, 0], [1, 0], [1, 0], [1, 0], [1, 1]],
                            eps=[[1, 0, 0, 0, 0]] * 4 + [[0, 0, 0, 0, 1]], boson=[0, 1]),
     (1.0, -0.3, 0.2, np.pi / 3, np.pi / 5), 2.0, W.real_axis(-3.0, 3.0, 5, 0.1)),
]


def setup(case):
    name, spec, lat, beta, X = case
    if spec == "bench":
        d = order4_bench()
        alpha, eps, boson, pref = d["alpha"], d["eps"], None, 1.0
    elif isinstance(spec, dict):
        alpha, eps, boson, pref = np.array(spec["alpha"]), spec["eps"], spec["boson"], 1.0
    else:
        d = O.enumerate_sigma(spec[0])[spec[1]]
        alpha, eps, boson, pref = d["alpha"], d["eps"], None, (-1.0) ** spec[0] * (-1.0) ** d["loops"]
    D = T.Diagram(alpha, eps=eps, var_is_boson=boson, prefactor=pref).upload(0)
    S = O.Solution(alpha, eps=eps, var_is_boson=boson, prefactor=pref)
    return D, S, lat, beta, X


def families_agree(S, lat, seed, off, X, beta, g, r0, r1, n_check=2000):
    """Reduced outputs of two kernel families over the same samples, whose per-sample values the
    families round differently (the specialised kernels sum the pole DAG's contributions in other
    orders, form the frequency loop's products on the integer pipes and fuse fewer products into
    fmas): the means, dSigma/dX and the gradients to the mean of the per-sample differences plus
    the rounding of the sums, the variances to the rounding of the sums -- and the per-sample
    derivative differences, on a prefix, within twice the oracle's derivative-envelope bound
    (once per side)."""
    m0, v0, p0, b0 = r0
    m1, v1, p1, b1 = r1
    scale = p0.abs().mean(dim=1)
    assert torch.all((m1 - m0).abs() <= (p1 - p0).abs().mean(dim=1) + 1e-12 * scale)
    assert torch.allclose(v1, v0, rtol=1e-10, atol=0)
    for red, per in (("dSigma_dX", "dX"), ("grad_params", "grads")):
        dim = 1 if per == "dX" else 0
        spread = (b1[per] - b0[per]).abs().mean(dim=dim)
        assert torch.all((b1[red] - b0[red]).abs() <= spread + 1e-12 * b0[per].abs().mean(dim=dim)), red
    k = min(n_check, b0["grads"].shape[0])
    _, dref, denv = S.eval_momenta_deriv(lat, seed, off, k, X, beta, "omega", threads=8, envelope=True)
    assert np.all(np.abs(b1["dX"][:, :k].cpu().numpy() - b0["dX"][:, :k].cpu().numpy()) <= 2 * RTOL * denv)
    for j, which in enumerate(("mu", "kx", "ky")):
        _, der, env = S.eval_momenta_deriv(lat, seed, off, k, X, beta, which, threads=8, envelope=True)
        bound = 2 * RTOL * (np.abs(g)[:, None] * env).sum(axis=0)
        diff = np.abs(b1["grads"][:k, j].cpu().numpy() - b0["grads"][:k, j].cpu().numpy())
        assert np.all(diff <= bound), which


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_specialised_kernel_against_oracle(case):
    """Every sample's value, dSigma/dX and contracted gradients from the specialised kernel against
    the oracle (values, forward-mode dual numbers), over several tiles and a ragged tail."""
    D, S, lat, beta, X = setup(case)
    T.set_jit("always")
    n, seed, off = 3 * 128 + 37, 21, 5
    g = upstream(len(X))
    out = D.forward_backward(lat, seed, off, n, X, beta, g, per_sample=True)
    torch.cuda.synchronize()
    st = D.jit_status()
    assert st["ready"] and st["last_used"] and st["compile_ms"] > 0
    ref = S.eval_momenta(lat, seed, off, n, X, beta, per_sample=True, threads=8)
    v = out["values"].cpu().numpy()
    vb = Bd.value_bound(ref, lat)
    assert np.all(np.abs(v - ref["values"]) <= vb), np.max(np.abs(v - ref["values"]) / vb)
    dref, dbd = Bd.oracle_deriv(S, lat, seed, off, n, X, beta, "omega")
    dX = out["dX"].cpu().numpy()
    assert np.all(np.abs(dX - dref) <= dbd), np.max(np.abs(dX - dref) / dbd)
    grads = out["grads"].cpu().numpy()
    for k, which in enumerate(("mu", "kx", "ky")):
        der, env = Bd.oracle_deriv(S, lat, seed, off, n, X, beta, which)
        gref = np.real(np.conj(g)[:, None] * der).sum(axis=0)
        bound = (np.abs(g)[:, None] * env).sum(axis=0)
        assert np.all(np.abs(grads[:, k] - gref) <= bound), (which, np.max(np.abs(grads[:, k] - gref) / bound))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_specialised_kernel_agrees_with_generic(case):
    """The specialised and the generic kernel on the same samples: reduced outputs agree to the
    rounding of the sums, and a second specialised run gives the same bits."""
    D, S, lat, beta, X = setup(case)
    n, seed, off = 5000, 7, 1 << 33
    g = upstream(len(X), seed=9)
    T.set_jit("never")
    gen = D.forward_backward(lat, seed, off, n, X, beta, g, per_sample=True)
    torch.cuda.synchronize()
    assert not D.jit_status()["last_used"]
    T.set_jit("always")
    jit = D.forward_backward(lat, seed, off, n, X, beta, g, per_sample=True)
    again = D.forward_backward(lat, seed, off, n, X, beta, g, per_sample=True)
    torch.cuda.synchronize()
    assert D.jit_status()["last_used"]
    for k in ("mean", "var", "dSigma_dX", "grad_params", "values", "dX", "grads"):
        assert torch.equal(jit[k], again[k]), k
    families_agree(S, lat, seed, off, X, beta, g, (gen["mean"], gen["var"], gen["values"], gen),
                   (jit["mean"], jit["var"], jit["values"], jit))


@pytest.mark.parametrize("n", [1, 2, 511, 512, 513, 1537])
def test_specialised_kernels_at_tile_edges(n):
    """The Monte Carlo kernels run 512-sample tiles in lockstep blocks (every lane reaches every
    barrier; a lane past the end runs the last sample again and adds and writes nothing).  At
    sample counts around the tile size: the fused pass's and the forward's per-sample outputs equal
    those of a longer launch over the same samples bit for bit, and the reduced outputs are the
    means (and the variance) of the per-sample ones."""
    D, S, lat, beta, X = setup(CASES[2])
    T.set_jit("always")
    seed, off = 13, 77
    g = upstream(len(X), seed=4)
    big = D.forward_backward(lat, seed, off, 2048, X, beta, g, per_sample=True)
    out = D.forward_backward(lat, seed, off, n, X, beta, g, per_sample=True)
    m, v, ps = D.forward(lat, seed, off, n, X, beta, per_sample=True)
    torch.cuda.synchronize()
    assert D.jit_status()["last_used"]
    assert torch.equal(out["values"], big["values"][:, :n]) and torch.equal(ps, big["values"][:, :n])
    assert torch.equal(out["dX"], big["dX"][:, :n]) and torch.equal(out["grads"], big["grads"][:n])
    p = ps.cpu().numpy()
    scale = np.abs(p).mean(axis=1)
    for mean in (m.cpu().numpy(), out["mean"].cpu().numpy()):
        assert np.all(np.abs(mean - p.mean(axis=1)) <= 1e-13 * scale)
    if n > 1:
        var = np.stack([np.var(p.real, axis=1, ddof=1), np.var(p.imag, axis=1, ddof=1)], axis=1)
        for vv in (v.cpu().numpy(), out["var"].cpu().numpy()):
            assert np.allclose(vv, var, rtol=1e-9, atol=1e-300)
    dX = out["dX"].cpu().numpy()
    assert np.all(np.abs(out["dSigma_dX"].cpu().numpy() - dX.mean(axis=1)) <= 1e-13 * np.abs(dX).mean(axis=1))
    gr = out["grads"].cpu().numpy()
    assert np.all(np.abs(out["grad_params"].cpu().numpy() - gr.mean(axis=0)) <= 1e-13 * np.abs(gr).mean(axis=0))


def test_auto_mode_takes_the_specialised_kernel_for_large_launches():
    """auto (the default): the generic kernel below 2^21 samples, the specialised one from there on
    (compiled on that first call and kept with the diagram)."""
    d = order4_bench()
    D = T.Diagram(d["alpha"], eps=d["eps"]).upload(0)
    c = W.ORDER4
    X, g = W.matsubara(c["beta"], c["n_freq"]), np.ones(c["n_freq"]) + 0.5j
    T.set_jit("auto")
    D.forward_backward(W.lattice(c), c["seed"], 0, 4096, X, c["beta"], g)
    torch.cuda.synchronize()
    st = D.jit_status()
    assert not st["ready"] and not st["last_used"]
    out = D.forward_backward(W.lattice(c), c["seed"], 0, 1 << 21, X, c["beta"], g)
    torch.cuda.synchronize()
    st = D.jit_status()
    assert st["ready"] and st["last_used"]
    assert np.all(np.isfinite(out["mean"].cpu().numpy()))
    T.set_jit("never")
    D.forward_backward(W.lattice(c), c["seed"], 0, 1 << 21, X, c["beta"], g)
    torch.cuda.synchronize()
    assert not D.jit_status()["last_used"]


def test_two_externals_build_the_energy_kernel_only():
    """A two-external diagram has no Monte Carlo calls (they need one external momentum):
    tami_jit_prepare builds its energy-input kernel only, and the fused call is refused
    (TAMI_EUNSUPPORTED) in every mode."""
    D = T.Diagram([[1, 1, 0], [1, 0, 1]], n_ext=2).upload(0)
    T.set_jit("always")
    D.jit_prepare()
    assert D.jit_status()["ready"] == {"energy"}
    with pytest.raises(L.TamiError) as e:
        D.forward_backward((1.0, 0.0, 0.0, 0.5, 0.5), 1, 0, 256, np.array([1j * np.pi]), 1.0, np.ones(1) + 0j)
    assert e.value.code == L.TAMI_EUNSUPPORTED


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_specialised_forward_and_adjoint_against_oracle(case):
    """The two-call path on the specialised kernels: the forward (keeping the saved rows) against the
    oracle's values, its saved rows equal to the generic forward's bit for bit, and the adjoint --
    reading those rows and recomputing -- against the oracle's dual numbers."""
    D, S, lat, beta, X = setup(case)
    n, seed, off = 3 * 128 + 37, 13, 2
    g = upstream(len(X), seed=4)
    T.set_jit("never")
    sv_gen = D.saved_buffer(n)
    D.forward(lat, seed, off, n, X, beta, save=sv_gen)
    T.set_jit("always")
    sv = D.saved_buffer(n)
    mean, var, ps = D.forward(lat, seed, off, n, X, beta, per_sample=True, save=sv)
    torch.cuda.synchronize()
    assert D.jit_status()["last_used"] and "forward" in D.jit_status()["ready"]
    assert torch.equal(sv, sv_gen)
    ref = S.eval_momenta(lat, seed, off, n, X, beta, per_sample=True, threads=8)
    v = ps.cpu().numpy()
    assert np.all(np.abs(v - ref["values"]) <= Bd.value_bound(ref, lat))
    scale = Bd.mean_scale(ref, lat)
    assert np.all(np.abs(mean.cpu().numpy() - ref["mean"]) <= RTOL * scale)
    dref, denv = Bd.oracle_deriv(S, lat, seed, off, n, X, beta, "omega")
    for saved in (sv, None):
        b = D.backward(lat, seed, off, n, X, beta, g, per_sample=True, saved=saved)
        torch.cuda.synchronize()
        assert D.jit_status()["last_used"] and "adjoint" in D.jit_status()["ready"]
        dX = b["dX"].cpu().numpy()
        assert np.all(np.abs(dX - dref) <= denv), np.max(np.abs(dX - dref) / denv)
        grads = b["grads"].cpu().numpy()
        for k, which in enumerate(("mu", "kx", "ky")):
            der, env = Bd.oracle_deriv(S, lat, seed, off, n, X, beta, which)
            gref = np.real(np.conj(g)[:, None] * der).sum(axis=0)
            assert np.all(np.abs(grads[:, k] - gref) <= (np.abs(g)[:, None] * env).sum(axis=0)), which


def test_specialised_forward_and_adjoint_agree_with_generic():
    """Bench table, 1e5 samples: reduced forward and adjoint outputs of the specialised kernels
    against the generic kernels'."""
    D, S, lat, beta, X = setup(CASES[2])
    n, seed, off = 100_000, 3, 0
    g = np.ones(len(X)) + 0.5j
    out = {}
    for mode in ("never", "always"):
        T.set_jit(mode)
        sv = D.saved_buffer(n)
        m, v, ps = D.forward(lat, seed, off, n, X, beta, per_sample=True, save=sv)
        b = D.backward(lat, seed, off, n, X, beta, g, per_sample=True, saved=sv)
        torch.cuda.synchronize()
        assert D.jit_status()["last_used"] == (mode == "always")
        out[mode] = (m, v, ps, b)
    families_agree(S, lat, seed, off, X, beta, g, out["never"], out["always"])


ENERGY_CASES = [
    # name, alpha, eps, boson, n_ext
    ("paper_order2", [[1, 0, 0], [0, 1, 0], [-1, 1, 1]], None, None, 1),
    ("order4_bench", "bench", None, None, 1),
    ("two_fermionic_ext", [[1, 1, 0], [1, 0, 1]], None, None, 2),
    ("three_externals", [[1, 1, 0, 0], [1, 0, 1, 0], [1, 0, 0, 1]], None, [0, 1, 0, 0], 3),
    ("order4_held_external", "held", None, None, 2),
]


@pytest.mark.parametrize("real_axis", [False, True], ids=["matsubara", "real_axis"])
@pytest.mark.parametrize("case", ENERGY_CASES, ids=[c[0] for c in ENERGY_CASES])
def test_specialised_energy_input_against_oracle(case, real_axis):
    """The energy-input kind: every (frequency row, energy row) value against the oracle, with one,
    two and three external frequencies, on the imaginary axis and with the first external
    continued to omega + i Gamma; and against the generic kernel."""
    name, alpha, eps, boson, n_ext = case
    if alpha == "bench":
        d = order4_bench()
        alpha, eps = d["alpha"], d["eps"]
    elif alpha == "held":
        d = order4_bench()
        alpha, eps = W.hold_external(d["alpha"], 3), d["eps"]
    alpha = np.asarray(alpha)
    D = T.Diagram(alpha, eps=eps, var_is_boson=boson, n_ext=n_ext).upload(0)
    S = O.Solution(alpha, eps=eps, var_is_boson=boson, n_ext=n_ext)
    beta = 2.0
    bext = [0] * n_ext if boson is None else list(boson[-n_ext:])
    X = np.empty((6, n_ext), dtype=np.complex128)
    for q, b in enumerate(bext):
        nn = np.arange(6) * (q + 1) - 2 * q + (1 if b else 0)
        X[:, q] = 1j * (2 * nn + (0 if b else 1)) * np.pi / beta
    if real_axis:
        X[:, 0] = np.linspace(-2.0, 2.0, 6) + 0.05j
    if n_ext == 1:
        X = X[:, 0]
    E = W.random_energies(3 * 128 + 37, alpha.shape[0], a=4.0, seed=17)
    Ed = torch.tensor(E, device="cuda")
    T.set_jit("always")
    out = D.eval_energies(Ed, X, beta)
    torch.cuda.synchronize()
    assert D.jit_status()["last_used"] and "energy" in D.jit_status()["ready"]
    ref, _, env = S.eval_energies(E, X, beta)
    got = out.cpu().numpy()
    assert np.all(np.abs(got - ref) <= RTOL * env), np.max(np.abs(got - ref) / env)
    T.set_jit("never")
    gen = D.eval_energies(Ed, X, beta).cpu().numpy()
    assert np.all(np.abs(got - gen) <= RTOL * env)


FALLBACK_SCRIPT = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import _lib as L, workloads as W
torch.cuda.set_device(0)
d = next(x for x in T.enumerate_sigma(4) if x["code"] == tuple(W.ORDER4["code"]))
D = T.Diagram(d["alpha"], eps=d["eps"]).upload(0)
c = W.ORDER4
X, g = W.matsubara(c["beta"], 4), np.ones(4) + 0.5j
out = {}
T.set_jit("auto")
r = D.forward_backward(W.lattice(c), c["seed"], 0, 1 << 21, X, c["beta"], g)
torch.cuda.synchronize()
out["auto_finite"] = bool(np.all(np.isfinite(r["mean"].cpu().numpy())))
out["auto_used"] = D.jit_status()["last_used"]
T.set_jit("always")
try:
    D.forward_backward(W.lattice(c), c["seed"], 0, 1024, X, c["beta"], g)
    out["always"] = "ran"
except L.TamiError as e:
    out["always"] = [e.code, str(e)]
T.set_jit("never")
r2 = D.forward_backward(W.lattice(c), c["seed"], 0, 1 << 21, X, c["beta"], g)
torch.cuda.synchronize()
out["same_as_generic"] = bool(torch.equal(r["mean"], r2["mean"]))
T.set_jit("auto")
B = T.Batch([D], [1 << 20], [c["seed"]], len(X), chunk_tiles=4)
out["batch_auto_specialised"] = B.info()["specialised"]
m, _ = B.launch(W.lattice(c), X, c["beta"])
torch.cuda.synchronize()
out["batch_auto_finite"] = bool(torch.isfinite(torch.view_as_real(m)).all())
T.set_jit("always")
try:
    T.Batch([D], [1 << 20], [c["seed"]], len(X), chunk_tiles=4)
    out["batch_always"] = "planned"
except L.TamiError as e:
    out["batch_always"] = [e.code, str(e)]
print(json.dumps(out))
"""


def test_without_nvrtc_auto_falls_back_and_always_refuses(tmp_path):
    """Failure of the run-time compiler, made on the host ($TAMI_NVRTC=none, in a child process):
    `auto` runs the generic kernel (the same bits as `never`) and plans batches on the persistent
    kernel alone, `always` refuses the call and the plan with TAMI_EUNSUPPORTED and says why, and
    nothing faults."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "fallback.py"
    script.write_text(FALLBACK_SCRIPT)
    env = dict(os.environ, TAMI_NVRTC="none")
    r = subprocess.run([sys.executable, str(script), root], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["auto_finite"] and not out["auto_used"] and out["same_as_generic"]
    assert out["always"][0] == L.TAMI_EUNSUPPORTED and "NVRTC disabled" in out["always"][1]
    assert out["batch_auto_specialised"] == 0 and out["batch_auto_finite"]
    assert out["batch_always"][0] == L.TAMI_EUNSUPPORTED and "NVRTC disabled" in out["batch_always"][1]


CACHE_SCRIPT = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import workloads as W
torch.cuda.set_device(0)
d = next(x for x in T.enumerate_sigma(4) if x["code"] == tuple(W.ORDER4["code"]))
D = T.Diagram(d["alpha"], eps=d["eps"]).upload(0)
c = W.ORDER4
X, g = W.matsubara(c["beta"], 4), np.ones(4) + 0.5j
D.jit_prepare()
st = D.jit_status()
T.set_jit("always")
r = D.forward_backward(W.lattice(c), c["seed"], 0, 4096, X, c["beta"], g)
torch.cuda.synchronize()
bits = [float(v).hex() for v in torch.view_as_real(r["mean"]).cpu().numpy().ravel()]
bits += [float(v).hex() for v in r["grad_params"].cpu().numpy().ravel()]
print(json.dumps({"ready": sorted(st["ready"]), "cached": sorted(st["cached"]), "bits": bits}))
"""


def test_disk_cache_of_compiled_kernels(tmp_path):
    """Compiled kernels persist across processes: a first process compiles and writes one entry
    per kind (no temporary file left), a second loads every kind from the cache and gives the same
    bits; a truncated entry is compiled again and rewritten; $TAMI_JIT_CACHE=none writes nothing."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "cache.py"
    script.write_text(CACHE_SCRIPT)
    cache, home = tmp_path / "cache", tmp_path / "home"
    home.mkdir()

    def run(cache_env):
        env = dict(os.environ, TAMI_JIT_CACHE=cache_env, HOME=str(home))
        r = subprocess.run([sys.executable, str(script), root], env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        return json.loads(r.stdout.strip().splitlines()[-1])

    first = run(str(cache))
    assert first["ready"] == ["adjoint", "energy", "forward", "fused"] and first["cached"] == []
    entries = sorted(cache.iterdir())
    assert len(entries) == 4 and all(p.suffix == ".tjc" for p in entries)
    second = run(str(cache))
    assert second["cached"] == second["ready"] == first["ready"]
    assert second["bits"] == first["bits"]
    size = entries[0].stat().st_size
    with open(entries[0], "r+b") as f:
        f.truncate(size // 2)
    third = run(str(cache))
    assert len(third["cached"]) == 3 and third["bits"] == first["bits"]
    assert entries[0].stat().st_size == size and len(list(cache.iterdir())) == 4
    off = run("none")
    assert off["cached"] == [] and off["bits"] == first["bits"]
    assert not any(home.rglob("*.tjc"))


@pytest.mark.parametrize("mode", ["always", "never"])
def test_every_enumerated_diagram(mode):
    """Every Hubbard self-energy diagram of orders 2-5 (85 tables, up to 744 flat terms) through
    the fused forward + adjoint kernel and through the two-call path (forward keeping rows, adjoint
    reading them): each sample's value, dSigma/dX and contracted gradients against the oracle, over
    a tile and a ragged tail; half of the diagrams on the imaginary axis
    and half on the real axis (the two phase-2 variants).  Also each diagram's energy-input
    kernel against the oracle's energy-input evaluation.  "always": the diagrams' specialised
    kernels (compiled on parallel host threads first); "never": the generic kernels."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    diags = [(m, d) for m in (2, 3, 4, 5) for d in O.enumerate_sigma(m)]
    assert len(diags) == 85
    pref = [(-1.0) ** m * (-1.0) ** d["loops"] for m, d in diags]
    lib = [T.Diagram(d["alpha"], eps=d["eps"], prefactor=p).upload(0) for (m, d), p in zip(diags, pref)]
    if mode == "always":
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
            list(ex.map(lambda D: D.jit_prepare(), lib))
    T.set_jit(mode)
    lat, beta, n, off = (1.0, -0.2, 0.1, np.pi / 2, np.pi / 3), 5.0, 128 + 22, 7
    rng = np.random.default_rng(29)
    for i, ((m, d), p, D) in enumerate(zip(diags, pref, lib)):
        S = O.Solution(d["alpha"], eps=d["eps"], prefactor=p)
        X = W.matsubara(beta, 3) if i % 2 == 0 else W.real_axis(-2.0, 2.0, 3, 0.1)
        g = upstream(len(X), seed=i)
        seed = 100 + i
        out = D.forward_backward(lat, seed, off, n, X, beta, g, per_sample=True)
        sv = D.saved_buffer(n)        # the two-call path: forward keeping rows, adjoint reading them
        _, _, ps = D.forward(lat, seed, off, n, X, beta, per_sample=True, save=sv)
        two = D.backward(lat, seed, off, n, X, beta, g, per_sample=True, saved=sv)
        E = rng.uniform(-3.0, 3.0, size=(40, np.asarray(d["eps"]).shape[1]))
        ev = D.eval_energies(torch.as_tensor(E, device="cuda"), X, beta)
        torch.cuda.synchronize()
        assert D.jit_status()["last_used"] == (mode == "always"), i
        tag = (m, d["code"])
        ref = S.eval_momenta(lat, seed, off, n, X, beta, per_sample=True, threads=8)
        for v in (out["values"].cpu().numpy(), ps.cpu().numpy()):
            assert np.all(np.abs(v - ref["values"]) <= Bd.value_bound(ref, lat)), tag
        dref, denv = Bd.oracle_deriv(S, lat, seed, off, n, X, beta, "omega")
        for r in (out, two):
            assert np.all(np.abs(r["dX"].cpu().numpy() - dref) <= denv), tag
        for k, which in enumerate(("mu", "kx", "ky")):
            der, env = Bd.oracle_deriv(S, lat, seed, off, n, X, beta, which)
            gref = np.real(np.conj(g)[:, None] * der).sum(axis=0)
            for r in (out, two):
                grads = r["grads"].cpu().numpy()
                assert np.all(np.abs(grads[:, k] - gref) <= (np.abs(g)[:, None] * env).sum(axis=0)), (tag, which)
        eref, _, eenv = S.eval_energies(E, X, beta)
        assert np.all(np.abs(ev.cpu().numpy() - eref) <= RTOL * eenv), tag

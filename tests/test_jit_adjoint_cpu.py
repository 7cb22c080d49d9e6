"""The specialised kernels checked on the host, for every table: the generated
statements of the pole DAG, the group weights and their adjoints are run as plain Python on random
inputs, and the adjoints they produce are compared with complex-step derivatives of the forward
statements they belong to.

With wb_t the adjoint of the phase-2 weight W2_t (an input of the reverse sweep), the sweep's
Fermi-value adjoints must be dL/dF_v and its combination adjoints dL/dx_u (through the real
reciprocals rr = 1/x and the complex denominators' real parts b = +-x), for L = sum_t wb_t W2_t(F, x)
+ sum_c bb_c b_c(x), bb_c the adjoint of b_c from the frequency loop; with x = c E the energy
adjoints must be dL/dE_j and mu's their sum.  This exercises the pole DAG's
shared and sign-flipped prefixes, the groups whose weight cancelled to zero, the products kept
from the forward and the sums that take their first term as an assignment, independently of the
GPU; the segment sums are left out there (the derivative values that feed them are set to zero).
A second test runs the whole frequency-free chain from the base energies -- combinations, the
generated Fermi/Bose segment code with its derivative values, the pole DAG and the weights -- and
checks the energy adjoints of the reverse sweep, segment sums included, against complex-step
derivatives with respect to each energy (planted sign errors in the segment sums, the first and
second derivatives and the energy coefficients are caught).  A third runs one frequency of the
generated loop, on and off the imaginary axis, and checks its weight and denominator adjoints and
dSigma/dX against complex-step derivatives of the loop's own value.  A fourth checks the generated
line momenta and energies against the diagram's momentum labels, and the last two the generated
value itself against the oracle's (its own construction, term by term) at the same energies: the
Monte Carlo kinds, and the energy-input kind with one or two external frequencies per row.  No GPU
needed."""
import cmath
import math
import re

import numpy as np
import pytest

import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import workloads as W


def _order6():
    """Order-6 tables: the first, the first with second derivatives (diagram 70) and the one with
    the most flat terms (the order-6 workload's)."""
    ds = T.enumerate_sigma(6)
    big = next(i for i, d in enumerate(ds) if d["code"] == tuple(W.ORDER6["code"]))
    return [(i, ds[i]) for i in (0, 70, big)]


ORDER6 = _order6()


def tables():
    out = [("order2_bosonic", T.Diagram(W.ORDER2["alpha"], var_is_boson=W.ORDER2["var_is_boson"])),
           ("quadruple_pole", T.Diagram([[1, 0], [1, 0], [1, 0], [1, 0], [1, 1]],
                                        eps=[[1, 0, 0, 0, 0]] * 4 + [[0, 0, 0, 0, 1]], var_is_boson=[0, 1]))]
    for m in (2, 3, 4, 5):
        for i, d in enumerate(T.enumerate_sigma(m)):
            out.append((f"order{m}_{i}", T.Diagram(d["alpha"], eps=d["eps"])))
    out += [(f"order6_{i}", T.Diagram(d["alpha"], eps=d["eps"])) for i, d in ORDER6]
    return out


QUAD = ([[1, 0], [1, 0], [1, 0], [1, 0], [1, 1]], [[1, 0, 0, 0, 0]] * 4 + [[0, 0, 0, 0, 1]], [0, 1])


def _value_tables():
    return ([("order2_bosonic", T.Diagram(W.ORDER2["alpha"], var_is_boson=W.ORDER2["var_is_boson"]),
              (W.ORDER2["alpha"], None, W.ORDER2["var_is_boson"])),
             ("quadruple_pole", T.Diagram(QUAD[0], eps=QUAD[1], var_is_boson=QUAD[2]), QUAD)] +
            [(f"order{m}_{i}", T.Diagram(d["alpha"], eps=d["eps"]), (d["alpha"], d["eps"], None))
             for m in (2, 3, 4, 5) for i, d in enumerate(T.enumerate_sigma(m))] +
            [(f"order6_{i}", T.Diagram(d["alpha"], eps=d["eps"]), (d["alpha"], d["eps"], None)) for i, d in ORDER6])


HEX = re.compile(r"-?0x[0-9a-f.]+p[+-]\d+")


def _python(section):
    """The generated statements of one section as Python (declarations dropped, shared-memory
    stores and barriers skipped, fma/imul_ftz/rcp as plain arithmetic)."""
    out = []
    for st in re.split(r"[;{}]", section):
        st = st.strip()
        if not st or st.startswith(("__syncthreads", "jsv[", "reinterpret_cast")):
            continue                                 # barriers, shared-memory and output stores
        st = re.sub(r"^(const )?(double2|double|bool) ", "", st)
        parts = [p.strip() for p in _split_commas(st)]
        for p in parts:
            if "=" not in p:
                continue                         # a declaration without a value
            p = HEX.sub(lambda m: repr(float.fromhex(m.group(0))), p)
            p = re.sub(r"\bimul_ftz\(|\bimul\(", "mul(", p)
            out.append(p)
    return "\n".join(out)


def _split_commas(s):
    out, depth, cur = [], 0, ""
    for ch in s:
        depth += ch == "("
        depth -= ch == ")"
        if ch == "," and depth == 0:
            out.append(cur)
            cur = ""
        else:
            cur += ch
    return out + [cur]


def sections(src):
    """(energy combinations, forward from the real reciprocals to the frequency loop, reverse
    sweep) of a generated fused kernel, as Python."""
    body = src[src.index("for (long long tile"):]
    c0 = body.index("    double x0 = ")
    combos = body[c0:body.index("    double sg0_g", c0)]
    a = body.index("const double rr0") if "const double rr0" in body else body.index("double W2_0")
    fwd = body[a:body.index("if (xr_zero) {")]
    r0 = body.index("double xbar0")
    rev = body[r0:body.index("if (act) {", r0)]
    fwd = re.sub(r"double (Wb2_\d+|bb\d+) = 0\.0;", "", fwd)     # the reverse sweep's inputs, set below
    return _python(combos), _python(fwd), _python(rev)


class Inputs(dict):
    """Every name the statements read without writing it: a fixed random value."""

    def __init__(self, rng, zero=()):
        super().__init__()
        self.rng, self.zero = rng, zero

    def __missing__(self, k):
        if k in FUNCS or k in ("fabs", "isneg", "cexp", "make_double2", "fermi_poly") or k.startswith("tami_seg_"):
            raise KeyError(k)                    # the arithmetic helpers come from the globals
        if any(k.startswith(z) for z in self.zero):
            v = 0.0
        elif k.startswith("x"):
            v = float(self.rng.uniform(0.5, 2.0)) * (1 if self.rng.random() < 0.5 else -1)
        else:
            v = float(self.rng.uniform(-1.0, 1.0))
        self[k] = v
        return v


FUNCS = {"fma": lambda a, b, c: a * b + c, "mul": lambda a, b: a * b, "rcp": lambda a: 1.0 / a}


def run(code, ns):
    exec(code, dict(FUNCS), ns)
    return ns


@pytest.mark.parametrize("kind", ["fused", "adjoint"])
@pytest.mark.parametrize("name,D", tables(), ids=[t[0] for t in tables()])
def test_reverse_sweep_equals_complex_step_derivatives(name, D, kind):
    combos, fwd, rev = sections(D.jit_source(kind))
    fwd_c, rev_c = compile(fwd, "fwd", "exec"), compile(combos + "\n" + fwd + "\n" + rev, "all", "exec")
    from_e = compile(combos + "\n" + fwd, "combos+fwd", "exec")
    rng = np.random.default_rng(7)
    base = Inputs(rng, zero=("fvd",))
    run(rev_c, base)                                   # every input drawn, the sweep run once
    w2 = sorted({k for k in base if re.fullmatch(r"W2_\d+", k)})
    bs = sorted({k for k in base if re.fullmatch(r"b\d+", k)})
    assert w2, name

    def loss(var, h, code=fwd_c):                      # the forward statements recompute every value
        ns = dict(base)
        ns[var] = base[var] + 1j * h
        run(code, ns)
        return (sum(base["Wb2_" + t[3:]] * ns[t] for t in w2) +
                sum(base["bb" + b[1:]] * ns[b] for b in bs))   # the complex denominators' real parts b

    h = 1e-30
    checked = 0
    for v in sorted(k for k in base if re.fullmatch(r"fv\d+", k)):
        d = loss(v, h).imag / h
        got = base.get("fvbar" + v[2:], 0.0)
        assert abs(got - d) <= 1e-12 * max(1.0, abs(d)), (name, v, got, d)
        checked += 1
    for x in sorted(k for k in base if re.fullmatch(r"x\d+", k)):
        d = loss(x, h).imag / h
        got = base.get("xbar" + x[1:], 0.0)
        assert abs(got - d) <= 1e-12 * max(1.0, abs(d)), (name, x, got, d)
    # the energy adjoints through the combinations x = c E, and mu's (dE_j/dmu = 1)
    total, scale = 0.0, 1.0
    for e in sorted(k for k in base if re.fullmatch(r"E\d+", k)):
        d = loss(e, h, from_e).imag / h
        got = base.get("Ebar" + e[1:], 0.0)
        assert abs(got - d) <= 1e-12 * max(1.0, abs(d)), (name, e, got, d)
        total += d
        scale += abs(d)                                # the sum may cancel to (near) zero
    assert abs(base["mub"] - total) <= 1e-12 * scale, (name, base["mub"], total)
    assert checked > 0


# ---- the whole frequency-free chain: energies -> combinations -> Fermi/Bose values and their
# derivatives -> pole DAG -> weights, and back

class _Pair:
    def __init__(self, x, y):
        self.x, self.y = x, y


def _re(v):
    return v.real if isinstance(v, complex) else v


def _exp(t):
    return cmath.exp(t) if isinstance(t, complex) else math.exp(t)


def _fermi_poly(k, g, h, beta):
    """d^k/dx^k of g at (g, h = 1 - g), written out from dg/dx = -beta g h (so an independent
    statement of the polynomials the kernels call)."""
    if k == 0:
        return g
    gh = g * h
    if k == 1:
        return -beta * gh
    if k == 2:
        return beta ** 2 * gh * (h - g)
    if k == 3:
        return -beta ** 3 * gh * ((h - g) ** 2 - 2 * gh)
    if k == 4:
        return beta ** 4 * gh * (h ** 3 - 11 * g * h * h + 11 * g * g * h - g ** 3)
    return -beta ** 5 * gh * (h ** 4 - 26 * g * h ** 3 + 66 * g * g * h * h - 26 * g ** 3 * h + g ** 4)


CHAIN_FUNCS = dict(FUNCS, fabs=lambda v: v if _re(v) >= 0 else -v, isneg=lambda v: _re(v) <= 0,
                   cexp=_exp, make_double2=_Pair, fermi_poly=_fermi_poly)


def _chain_python(section):
    """Segment code as Python as well: the exponential (e^t and e^t - 1), the sign test, selects."""
    out = []
    for line in _python(section).split("\n"):
        m = re.match(r"^y = exp_neg<\w+>\((.*), em\)$", line)
        if m:
            out += ["y = cexp(%s)" % m.group(1), "em = y - 1.0"]
            continue
        if line.startswith("(void)"):
            continue
        line = re.sub(r"__double_as_longlong\((\w+)\) <= 0", r"isneg(\1)", line)
        line = re.sub(r"(\w+) \? ([\w.]+) : ([\w.]+)", r"(\2 if \1 else \3)", line)
        out.append(line)
    return "\n".join(out)


def _device_functions(src):
    """The generated out-of-line segment functions (large tables) as Python functions."""
    code = []
    for m in re.finditer(r"double2 (tami_seg_\w+)\(double xv, double beta\) \{(.*?)\n\}", src, re.S):
        body = _chain_python(m.group(2).replace("return ", "ret = "))
        code.append("def %s(xv, beta):\n%s\n    return ret" % (
            m.group(1), "\n".join("    " + l for l in body.split("\n"))))
    return "\n".join(code)


def chain_sections(src):
    body = src[src.index("for (long long tile"):]
    c0 = body.index("    double x0 = ")
    fwd = body[c0:body.index("if (xr_zero) {")]
    fwd = re.sub(r"double (Wb2_\d+|bb\d+) = 0\.0;", "", fwd)
    r0 = body.index("double xbar0")
    rev = body[r0:body.index("if (act) {", r0)]
    return _chain_python(fwd), _python(rev)


@pytest.mark.parametrize("kind", ["fused", "adjoint"])
@pytest.mark.parametrize("name,D", tables(), ids=[t[0] for t in tables()])
def test_energy_adjoints_equal_complex_step_derivatives(name, D, kind):
    """With the Fermi/Bose values and their derivatives computed by the generated segment code from
    the energies, the energy adjoints of the reverse sweep (the segment sums included) equal
    complex-step derivatives of L = sum_t wb_t W2_t + sum_c bb_c b_c with respect to each base
    energy, and mu's adjoint their sum; random energies, beta, wb and bb.  Both kinds that carry
    the reverse sweep: the fused pass and the adjoint reading saved energies."""
    src = D.jit_source(kind)
    fwd, rev = chain_sections(src)
    glb = dict(CHAIN_FUNCS)
    exec(_device_functions(src), glb)
    fwd_c, all_c = compile(fwd, "fwd", "exec"), compile(fwd + "\n" + rev, "all", "exec")
    rng = np.random.default_rng(11)
    base = Inputs(rng)
    base["beta"] = float(rng.uniform(0.5, 2.0))
    for j in range(16):
        base["E%d" % j] = float(rng.uniform(-2.0, 2.0))
    exec(all_c, dict(glb), base)
    w2 = sorted({k for k in base if re.fullmatch(r"W2_\d+", k)})
    bs = sorted({k for k in base if re.fullmatch(r"b\d+", k)})

    def loss(var, h):
        ns = dict(base)
        ns[var] = base[var] + 1j * h
        exec(fwd_c, dict(glb), ns)
        return (sum(base["Wb2_" + t[3:]] * ns[t] for t in w2) + sum(base["bb" + b[1:]] * ns[b] for b in bs))

    h = 1e-30
    total, scale, checked = 0.0, 1.0, 0
    for e in sorted(k for k in base if re.fullmatch(r"E\d+", k) and "Ebar" + k[1:] in base):
        d = loss(e, h).imag / h
        got = base["Ebar" + e[1:]]
        assert abs(got - d) <= 1e-11 * max(1.0, abs(d)), (name, e, got, d)
        total += d
        scale += abs(d)
        checked += 1
    assert checked > 0
    assert abs(base["mub"] - total) <= 1e-11 * scale, (name, base["mub"], total)


# ---- the frequency loop: one frequency of the generated loop body

def _neg_rewrite(s):
    """The generated sign flip __longlong_as_double(__double_as_longlong(e) ^ sign bit) as -(e)."""
    head = "__longlong_as_double(__double_as_longlong("
    tail = ") ^ (long long)0x8000000000000000ull)"
    while head in s:
        i = s.index(head)
        j = _closing_paren(s, i + len(head) - 1)
        assert s[j:j + len(tail)] == tail, s[j:j + 60]
        s = s[:i] + "(-(" + s[i + len(head):j] + "))" + s[j + len(tail):]
    return s


def _closing_paren(s, i):
    depth = 0
    for j in range(i, len(s)):
        depth += s[j] == "("
        depth -= s[j] == ")"
        if depth == 0:
            return j
    raise AssertionError("unbalanced")


def loop_bodies(src):
    """(imaginary-axis body, general body, loop inputs as Python, shared-memory slot names) of the
    fused kernel's frequency loop."""
    body = src[src.index("for (long long tile"):]
    a = body.index("if (xr_zero) {")
    out = []
    for start in (a, body.index("} else {", a)):
        k = body.index("for (int f = 0; f < n_f; ++f) {", start)
        o = k + len("for (int f = 0; f < n_f; ++f) ")      # the loop's opening brace
        text = body[o + 1:_closing_brace(body, o)]
        text = re.sub(r"if \(act\) \{.*?\n\s*\}", "", text, flags=re.S)     # the running sums
        text = _neg_rewrite(text)
        text = text.replace("Xs[2 * f]", "Xr_in").replace("Gs[2 * f + 1]", "Gi_in").replace("Gs[2 * f]", "Gr_in")
        text = re.sub(r"Xs\[2 \* \((\d+) \* n_f \+ f\)\]", r"Yr_in_\1", text)   # energy input: Re Y_k
        text = re.sub(r"AXI2\[(\d+) \* n_f \+ f\]", r"AXI2_\1", text)
        text = re.sub(r"AXI\[(\d+) \* n_f \+ f\]", r"AXI_\1", text)
        text = re.sub(r"jsv\[(\d+) \* \d+ \+ tid\]", r"jsv_\1", text)
        out.append(_python(text))
    fwd = body[:a]
    pw = "\n".join(_python(m.group(0)) for m in re.finditer(r"const double pW\d+ = [^;]+;", fwd))
    slots = {int(m.group(1)): m.group(2) for m in re.finditer(r"jsv\[(\d+) \* \d+ \+ tid\] = (\w+);", fwd)}
    return out[0], out[1], pw, slots


def _closing_brace(s, i):
    depth = 0
    for j in range(i, len(s)):
        depth += s[j] == "{"
        depth -= s[j] == "}"
        if depth == 0:
            return j
    raise AssertionError("unbalanced")


@pytest.mark.parametrize("name,D", tables(), ids=[t[0] for t in tables()])
def test_frequency_loop_adjoints_equal_complex_step_derivatives(name, D):
    """One frequency of the generated loop, on and off the imaginary axis: with L = Re(conj(g) v)
    for the sample's value v = sum_t W2_t R_t(X) and an upstream gradient g, the loop's weight and
    denominator adjoints (Wb2, bb) equal complex-step derivatives of L with respect to W2 and to the
    denominators' real parts b, and its dv/dX equals the complex derivative of v (along the real
    axis, or i times the derivative along the imaginary one)."""
    src = D.jit_source("fused")
    on_axis, off_axis, pw, slots = loop_bodies(src)
    cden_a = [float.fromhex(v.strip()) for v in
              re.search(r"kJitCdenA\[\d+\] = \{([^}]*)\}", src).group(1).split(",")]
    rng = np.random.default_rng(5)
    text = "\n".join([pw] + list(slots.values()) + [on_axis])
    w2 = sorted(set(re.findall(r"\bW2_\d+\b", text)))
    bs = sorted(set(re.findall(r"\bb\d+\b", text)))
    vals = {k: float(rng.uniform(-1, 1)) for k in w2}
    vals.update({k: float(rng.uniform(0.5, 2.0)) * (1 if rng.random() < 0.5 else -1) for k in bs})
    Gr, Gi, Xr0, Xi0 = (float(v) for v in rng.uniform(-1, 1, 4))

    def run_body(body, v, Xr, Xi):
        ns = dict(v)
        ns.update(Gr_in=Gr, Gi_in=Gi, Xr_in=Xr)
        for c, a in enumerate(cden_a):
            ns["AXI_%d" % c], ns["AXI2_%d" % c] = a * Xi, (a * Xi) ** 2
        for k in [n for n in list(ns) if n.startswith(("Wb2_", "bb"))]:
            del ns[k]
        for t in w2:
            ns["Wb2_" + t[3:]] = 0.0
        for c in range(len(cden_a)):
            ns["bb%d" % c] = 0.0
        code = pw + "\n" + "\n".join("jsv_%d = %s" % (k, n) for k, n in sorted(slots.items())) + "\n" + body
        exec(code, dict(FUNCS), ns)
        return ns

    h = 1e-30
    for axis, body, Xr in (("on", on_axis, 0.0), ("off", off_axis, Xr0)):
        base = run_body(body, vals, Xr, Xi0)
        L = lambda ns: Gr * ns["vr"] + Gi * ns["vi"]

        def step(var, Xr=Xr, Xi=Xi0):
            v = dict(vals)
            if var in v:
                v[var] = v[var] + 1j * h
            return run_body(body, v, Xr, Xi)

        for t in w2:
            d = L(step(t)).imag / h
            assert abs(base["Wb2_" + t[3:]] - d) <= 1e-12 * max(1.0, abs(d)), (name, axis, t)
        for b in bs:
            d = L(step(b)).imag / h
            assert abs(base["bb" + b[1:]] - d) <= 1e-12 * max(1.0, abs(d)), (name, axis, b)
        if axis == "off":                              # d/dXr of v
            ns = step(None, Xr=Xr + 1j * h)
            dr, di = ns["vr"].imag / h, ns["vi"].imag / h
        else:                                          # dv/dX = -i d/dXi of v
            ns = step(None, Xi=Xi0 + 1j * h)
            dr, di = ns["vi"].imag / h, -ns["vr"].imag / h
        scale = max(1.0, abs(dr), abs(di))
        assert abs(base["dvr"] - dr) <= 1e-12 * scale and abs(base["dvi"] - di) <= 1e-12 * scale, (name, axis)


# ---- the line momenta and energies of the generated prologue (step a2/a3)

def _line_energy(ax, ay, t, tp, mu):
    cx, cy = math.cos(ax), math.cos(ay)
    return mu + 2.0 * t * (cx + cy) + 4.0 * tp * cx * cy


@pytest.mark.parametrize("name,D,alpha", [(n, D, a) for n, D, a in
                                          [(t[0], t[1], None) for t in tables()[:1]] +
                                          [(f"order{m}_{i}", T.Diagram(d["alpha"], eps=d["eps"]), d["alpha"])
                                           for m in (2, 3, 4, 5) for i, d in enumerate(T.enumerate_sigma(m))]],
                         ids=lambda v: v if isinstance(v, str) else "")
def test_line_energies_follow_the_momentum_labels(name, D, alpha):
    """Every line energy the generated kernel computes is mu - eps(K_j) of the line's momentum
    K_j = sum_l alpha_jl k_l + alpha_j,ext k_ext, with the labels read from the diagram (not from
    the generated code), for random loop and external momenta and lattice parameters."""
    if alpha is None:
        alpha = np.array(W.ORDER2["alpha"])
    src = D.jit_source("fused")
    body = src[src.index("for (long long tile"):]
    m = alpha.shape[1] - 1
    a = body.index("const double kx%d = lkx" % m)
    prologue = body[a:body.index("\n    }", a)]
    prologue = re.sub(r"line_energy_grad\(([^,]+), ([^,]+), lt, ltp, lmu, \w+, \w+\)",
                      r"line_energy(\1, \2, lt, ltp, lmu)", prologue)
    code = _python(prologue.replace("(void)kx%d; (void)ky%d;" % (m, m), ""))
    rng = np.random.default_rng(3)
    ns = {"kx%d" % l: float(rng.uniform(-np.pi, np.pi)) for l in range(m)}
    ns.update({"ky%d" % l: float(rng.uniform(-np.pi, np.pi)) for l in range(m)})
    ns.update(lkx=float(rng.uniform(-np.pi, np.pi)), lky=float(rng.uniform(-np.pi, np.pi)),
              lt=1.0, ltp=float(rng.uniform(-0.5, 0.5)), lmu=float(rng.uniform(-1, 1)))
    exec(code, {"fma": FUNCS["fma"], "line_energy": _line_energy}, ns)
    lines = sorted(int(k[1:]) for k in ns if re.fullmatch(r"E\d+", k))
    assert lines, name
    for j in lines:
        kx = sum(int(alpha[j][l]) * ns["kx%d" % l] for l in range(m)) + int(alpha[j][m]) * ns["lkx"]
        ky = sum(int(alpha[j][l]) * ns["ky%d" % l] for l in range(m)) + int(alpha[j][m]) * ns["lky"]
        want = _line_energy(kx, ky, ns["lt"], ns["ltp"], ns["lmu"])
        assert abs(ns["E%d" % j] - want) <= 1e-12, (name, j)


# ---- the generated value against the oracle, on the host

@pytest.mark.parametrize("kind", ["forward", "fused"])
@pytest.mark.parametrize("name,D,oracle_args", _value_tables(), ids=lambda v: v if isinstance(v, str) else "")
def test_generated_value_matches_the_oracle(name, D, oracle_args, kind):
    """The generated per-sample code from the base energies on -- combinations, the Fermi/Bose
    segments, the pole DAG, the weights and one frequency of the loop -- run as Python, gives the
    oracle's value of the same diagram (its own construction, term by term) at the same energies,
    on and off the imaginary axis, within 1e-12 of the oracle's rounding envelope."""
    import oracle as O
    src = D.jit_source(kind)
    fwd, _ = chain_sections(src) if kind == "fused" else (None, None)
    if kind == "forward":
        body = src[src.index("for (long long tile"):]
        c0 = body.index("    double x0 = ")
        fwd = _chain_python(body[c0:body.index("if (xr_zero) {")])
    on_axis, off_axis, pw, slots = loop_bodies(src)
    cden_a = [float.fromhex(v.strip()) for v in
              re.search(r"kJitCdenA\[\d+\] = \{([^}]*)\}", src).group(1).split(",")]
    glb = dict(CHAIN_FUNCS)
    exec(_device_functions(src), glb)
    alpha, eps, boson = oracle_args
    alpha = np.asarray(alpha)
    sol = O.Solution(alpha, eps=eps, var_is_boson=boson)
    rng = np.random.default_rng(13)
    rows = {}
    E = np.empty(alpha.shape[0])
    for j, row in enumerate(map(tuple, alpha)):          # lines with equal labels share an energy
        rows.setdefault(row, float(rng.uniform(-2.0, 2.0)))
        E[j] = rows[row]
    beta = 1.3
    for body, X in ((on_axis, complex(0.0, 3 * np.pi / beta)), (off_axis, complex(0.7, 0.05))):
        ns = {"E%d" % j: float(E[j]) for j in range(len(E))}
        ns.update(beta=beta, Xr_in=X.real, Gr_in=0.0, Gi_in=0.0)
        for c, a in enumerate(cden_a):
            ns["AXI_%d" % c], ns["AXI2_%d" % c] = a * X.imag, (a * X.imag) ** 2
        for k in range(64):
            ns["Wb2_%d" % k] = 0.0
            ns["bb%d" % k] = 0.0
        code = fwd + "\n" + "\n".join("jsv_%d = %s" % (k, n) for k, n in sorted(slots.items())) + "\n" + body
        exec(code, dict(glb), ns)
        want, _, env = sol.eval_energies(E[None, :], np.array([X]), beta)
        got = complex(ns["vr"], ns["vi"])
        assert abs(got - want[0, 0]) <= 1e-12 * env[0, 0] + 1e-300, (name, kind, X, got, want[0, 0])


FREQ_FREE = [[1, 0], [1, 0]]   # sum_nu G1 G2, no external frequency: R = 1 and one real denominator E1 - E2


def _energy_kind_tables():
    out = [(t[0], t[1], t[2], 1) for t in _value_tables()]
    out.append(("frequency_free", T.Diagram(FREQ_FREE), (FREQ_FREE, None, None), 1))
    for m, i in ((3, 0), (3, 1), (4, 0), (4, 5), (4, 11)):
        d = T.enumerate_sigma(m)[i]
        a2 = W.hold_external(d["alpha"], m - 1)
        out.append((f"order{m}_{i}_two_external", T.Diagram(a2, eps=d["eps"], n_ext=2), (a2, d["eps"], None), 2))
    return out


@pytest.mark.parametrize("name,D,oracle_args,n_ext", _energy_kind_tables(),
                         ids=lambda v: v if isinstance(v, str) else "")
def test_energy_kind_value_matches_the_oracle(name, D, oracle_args, n_ext):
    """The energy-input kind (energies read, every value written; several external frequencies per
    row): its generated per-row code, run as Python from the base energies with the frequency row
    staged as the kernel stages it (Y_k = sum_q v_kq X_q), gives the oracle's value at the same
    energies and frequency row, on and off the imaginary axis, within 1e-12 of its envelope."""
    import oracle as O
    src = D.jit_source("energy")
    body = src[src.index("for (long long tile"):]
    c0 = body.index("    double x0 = ")
    fwd = _chain_python(body[c0:body.index("if (xr_zero) {")])
    on_axis, off_axis, pw, slots = loop_bodies(src)
    m = re.search(r"kJitCdenA\[\d+\] = \{([^}]*)\}", src)
    cden_a = [float.fromhex(v.strip()) for v in m.group(1).split(",")] if m else []
    m = re.search(r"kJitCdenXk\[\d+\] = \{([^}]*)\}", src)
    cden_xk = [int(v) for v in m.group(1).split(",")] if m else [0] * len(cden_a)
    m = re.search(r"kJitXvec\[\d+\] = \{([^}]*)\}", src)
    xvec = (np.array([float.fromhex(v.strip()) for v in m.group(1).split(",")]).reshape(-1, n_ext)
            if m else np.ones((1, 1)))
    glb = dict(CHAIN_FUNCS)
    exec(_device_functions(src), glb)
    alpha, eps, boson = oracle_args
    alpha = np.asarray(alpha)
    sol = O.Solution(alpha, eps=eps, var_is_boson=boson, n_ext=n_ext)
    rng = np.random.default_rng(17)
    E = rng.uniform(-2.0, 2.0, alpha.shape[0])         # energy input: every line its own energy
    beta = 1.1
    on = np.array([1j * np.pi * (2 * q + 1) / beta for q in range(n_ext)])
    off = np.array([0.6 - 0.3 * q + 0.04j for q in range(n_ext)])
    for body_code, Xrow in ((on_axis, on), (off_axis, off)):
        Y = xvec @ Xrow
        ns = {"E%d" % j: float(E[j]) for j in range(len(E))}
        ns.update(beta=beta, Xr_in=0.0)
        for k, y in enumerate(Y):
            ns["Yr_in_%d" % k] = y.real
        for c, (a, k) in enumerate(zip(cden_a, cden_xk)):
            ns["AXI_%d" % c], ns["AXI2_%d" % c] = a * Y[k].imag, (a * Y[k].imag) ** 2
        exec(fwd + "\n" + body_code, dict(glb), ns)
        want, _, env = sol.eval_energies(E[None, :], Xrow[None, :], beta)
        got = complex(ns["vr"], ns["vi"])
        assert abs(got - want[0, 0]) <= 1e-12 * env[0, 0] + 1e-300, (name, Xrow, got, want[0, 0])


def test_paper_order2_example_is_evaluated_in_factorised_form():
    """The paper's order-2 example (Sec. 5, the tree of its factorisation figure): its four flat
    terms A FT R share one denominator, and the generated pole DAG evaluates their Fermi part as a
    product of two differences of Fermi/Bose values, [F_a - F_b][F_c - F_d] (three arithmetic DAG
    steps), not as four products."""
    sympy = pytest.importorskip("sympy")
    D = T.Diagram(np.array([[1, 0, 0], [0, 1, 0], [-1, 1, 1]], dtype=np.int8))
    assert D.info()["n_terms"] == 4
    src = D.jit_source("forward")
    body = src[src.index("double W2_0"):src.index("const double b0")]     # the DAG and the weight
    fv = {v: sympy.Symbol(v) for v in set(re.findall(r"\bfv\d+\b", body))}
    ns = dict(fv)
    code = _python(body)
    exec(code, {"fma": lambda a, b, c: a * b + c, "mul": lambda a, b: a * b}, ns)
    w = sympy.expand(ns["W2_0"])
    assert len(w.as_ordered_terms()) == 4                         # the four flat terms
    factors = [f for f in sympy.factor_list(w)[1]]
    assert len(factors) == 2 and all(len(sympy.Poly(f, *fv.values()).terms()) == 2 and e == 1
                                      for f, e in factors)
    assert len(re.findall(r"const double pv\d+ = (?:fma|imul_ftz)\(", body)) == 3   # (a copy is free)

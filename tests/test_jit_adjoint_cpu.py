"""The specialised kernels' reverse sweep checked on the host, for every table: the generated
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
second derivatives and the energy coefficients are caught).  No GPU needed."""
import cmath
import math
import re

import numpy as np
import pytest

import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import workloads as W


def tables():
    out = [("order2_bosonic", T.Diagram(W.ORDER2["alpha"], var_is_boson=W.ORDER2["var_is_boson"])),
           ("quadruple_pole", T.Diagram([[1, 0], [1, 0], [1, 0], [1, 0], [1, 1]],
                                        eps=[[1, 0, 0, 0, 0]] * 4 + [[0, 0, 0, 0, 1]], var_is_boson=[0, 1]))]
    for m in (2, 3, 4, 5):
        for i, d in enumerate(T.enumerate_sigma(m)):
            out.append((f"order{m}_{i}", T.Diagram(d["alpha"], eps=d["eps"])))
    return out


HEX = re.compile(r"-?0x[0-9a-f.]+p[+-]\d+")


def _python(section):
    """The generated statements of one section as Python (declarations dropped, shared-memory
    stores and barriers skipped, fma/imul_ftz/rcp as plain arithmetic)."""
    out = []
    for st in re.split(r"[;{}]", section):
        st = st.strip()
        if not st or st.startswith("__syncthreads") or st.startswith("jsv["):
            continue
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


@pytest.mark.parametrize("name,D", tables(), ids=[t[0] for t in tables()])
def test_reverse_sweep_equals_complex_step_derivatives(name, D):
    combos, fwd, rev = sections(D.jit_source("fused"))
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


@pytest.mark.parametrize("name,D", tables(), ids=[t[0] for t in tables()])
def test_energy_adjoints_equal_complex_step_derivatives(name, D):
    """With the Fermi/Bose values and their derivatives computed by the generated segment code from
    the energies, the energy adjoints of the reverse sweep (the segment sums included) equal
    complex-step derivatives of L = sum_t wb_t W2_t + sum_c bb_c b_c with respect to each base
    energy, and mu's adjoint their sum; random energies, beta, wb and bb."""
    src = D.jit_source("fused")
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

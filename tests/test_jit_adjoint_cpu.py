"""The specialised kernels' reverse sweep checked on the host, for every table: the generated
statements of the pole DAG, the group weights and their adjoints are run as plain Python on random
inputs, and the adjoints they produce are compared with complex-step derivatives of the forward
statements they belong to.

With wb_t the adjoint of the phase-2 weight W2_t (an input of the reverse sweep), the sweep's
Fermi-value adjoints must be dL/dF_v and its real-denominator contributions to the combination
adjoints dL/dx_u (through rr = 1/x), for L = sum_t wb_t W2_t(F, x).  This exercises the pole DAG's
shared and sign-flipped prefixes, the groups whose weight cancelled to zero, the products kept
from the forward and the sums that take their first term as an assignment, independently of the
GPU; the segment sums and the energy adjoints are left out (the inputs that feed them, the
derivative values and the complex-denominator adjoints, are set to zero).  No GPU needed."""
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
        st = re.sub(r"^(const )?double ", "", st)
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
    body = src[src.index("for (long long tile"):]
    a = body.index("const double rr0") if "const double rr0" in body else body.index("double W2_0")
    fwd = body[a:body.index("if (xr_zero) {")]
    r0 = body.index("double xbar0")
    rev = body[r0:body.index("if (act) {", r0)]
    fwd = re.sub(r"double (Wb2_\d+|bb\d+) = 0\.0;", "", fwd)     # the reverse sweep's inputs, set below
    return _python(fwd), _python(rev)


class Inputs(dict):
    """Every name the statements read without writing it: a fixed random value."""

    def __init__(self, rng, zero=()):
        super().__init__()
        self.rng, self.zero = rng, zero

    def __missing__(self, k):
        if k in FUNCS:
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
    fwd, rev = sections(D.jit_source("fused"))
    fwd_c, rev_c = compile(fwd, "fwd", "exec"), compile(fwd + "\n" + rev, "fwd+rev", "exec")
    rng = np.random.default_rng(7)
    base = Inputs(rng, zero=("fvd", "bb"))
    run(rev_c, base)                                   # every input drawn, the sweep run once
    w2 = sorted({k for k in base if re.fullmatch(r"W2_\d+", k)})
    assert w2, name

    def loss(var, h):                                  # the forward statements recompute every value
        ns = dict(base)
        ns[var] = base[var] + 1j * h
        run(fwd_c, ns)
        return sum(base["Wb2_" + t[3:]] * ns[t] for t in w2)

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
    assert checked > 0

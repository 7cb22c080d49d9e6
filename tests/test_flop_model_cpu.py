"""The algorithmic flop model (tami_info.flops_per_sample and flops_per_sample_freq, which the
bench's roofline divides by time) counted a second way: from the forward kernel source the library
generates for the same table, statement by statement, under the model's conventions -- fma = 2,
mul or add = 1, a multiplication by +-1 or an addition to an exact 0 free, the reciprocal 6, the
exponential 19 (+2 for e^t - 1), a line energy 66 (two cosines of 30, then 6), the first
derivative -beta g h once per segment that needs it, the higher Fermi derivative polynomials as
listed below -- and with every sum written as an fma chain from 0
(line momenta, energy combinations, pole-DAG nodes) counted once per distinct prefix, since
chains that begin with the same steps share those partial sums.  No GPU needed: the source is
generated on the host."""
import re

import pytest

import paper_2311_17189_gb300 as T
from paper_2311_17189_gb300 import workloads as W

UNIT = ("0x1p+0", "-0x1p+0")
POLY = {0: 0, 1: 2, 2: 5, 3: 9, 4: 17, 5: 23}   # fermi_poly(k): g h, h - g, powers, the Eulerian sum


def step(first, coef):
    unit = coef in UNIT
    return (0 if unit else 1) if first else (1 if unit else 2)


def chains(body, pattern, start=None):
    """Flops of the fma chains `dst = fma(coef, var, dst)` (first step onto 0.0, or the chain
    started by `start`, a copy of +-var with no arithmetic), each distinct prefix once; pattern
    groups: dst, coef, var; start groups: dst, sign, var."""
    seen, cur, fl = {}, {}, 0
    if start:
        for m in re.finditer(start, body):
            pref = ((m.group(3), "-0x1p+0" if m.group(2) else "0x1p+0"),)
            seen[pref] = True
            cur[m.group(1)] = pref
    for m in re.finditer(pattern, body):
        dst, coef, var = m.group(1), m.group(2).strip(), m.group(3)
        first = dst not in cur
        pref = cur.get(dst, ()) + ((var, coef),)
        if pref not in seen:
            seen[pref] = True
            fl += step(first, coef)
        cur[dst] = pref
    return fl


def dag(body):
    """Pole-DAG prefixes: const double pv<k> = fma(fv<y>, OPERAND, 0.0 | pv<parent>), an operand
    being a leaf coefficient or another prefix (a node's value, possibly negated: a free operand
    sign); each written once."""
    fl, seen = 0, set()
    for m in re.finditer(r'const double pv(\d+) = (-?)fv(\d+);', body):   # +-F: a unit leaf, no arithmetic
        assert m.group(1) not in seen
        seen.add(m.group(1))
    for m in re.finditer(r'const double pv(\d+) = fma\(fv(\d+), ([^,]+), ([^)]+)\);', body):
        k, opnd, add = m.group(1), m.group(3).strip(), m.group(4).strip()
        assert k not in seen
        seen.add(k)
        fl += step(add == "0.0", "x" if opnd.lstrip("-").startswith("pv") else opnd)
    for m in re.finditer(r'const double pv(\d+) = imul_ftz\(fv(\d+), ([^)]+)\);', body):   # a first step,
        assert m.group(1) not in seen                                                     # on the integer pipes
        seen.add(m.group(1))
        fl += 1
    return fl


def per_sample(src):
    body = src[src.index("for (long long tile"):src.index("if (xr_zero) {")]
    fl = 2 * body.count("to_momentum(")
    fl += 2 * chains(body, r'ax(\d+) = fma\(([^,]+), kx(\d+), ax\d+\);',     # both components
                     r'double ax(\d+) = (-?)kx(\d+),')
    fl += 66 * len(re.findall(r'\bline_energy\(', body))                  # (the saved-rows branch aside)
    fl += chains(body, r'\bx(\d+) = fma\(([^,]+), E(\d+), x\d+\);', r'double x(\d+) = (-?)E(\d+);')
    bose = body.count("exp_neg<true>") + body.count("tami_seg_bose(")       # inline, or the out-of-line copy
    fermi = body.count("exp_neg<false>") + body.count("tami_seg_fermi(")     # that large tables call
    fl += (1 + 21 + 6 + 1) * bose                                           # -beta|x|, e^t and e^t - 1, 1/D, y/D
    fl += (1 + 19 + 7 + 1) * fermi                                          # ... D = 1 + y
    fl += sum(POLY[int(k)] for k in re.findall(r'fermi_poly\((\d+),', body))
    fl += 2 * len(re.findall(r'sg\d+_d1 = (?!0\.0;)', body))                 # -beta g h: the k = 1 values
    fl += 6 * len(re.findall(r'rr\d+ = rcp\(', body))
    fl += dag(body)
    # group weights: products on the FP64 unit (x *= y, x * y) or the integer pipes (imul_ftz(x, y))
    fl += len(re.findall(r'W1_\d+ (?:\*= rr\d+|= imul_ftz\(W1_\d+, rr\d+\));', body))
    fl += len(re.findall(r'W2_\d+ \+= W1_\d+;', body))
    fl += len(re.findall(r'RR_\d+ (?:\*= rr\d+|= imul_ftz\(RR_\d+, rr\d+\));', body))
    fl += len(re.findall(r'double W1_\d+ = (?:-?pv\d+ \* RR_\d+|imul_ftz\(-?pv\d+, RR_\d+\));', body))
    return fl


def per_frequency(src):
    a = src.index("if (xr_zero) {")
    loop = src[a:src.index("} else {", a)]
    fl = 10 * len(re.findall(r'= rcp\(fma\(Dr\d+, Dr\d+,', loop))          # |D|^2, reciprocal, 1/D
    fl += 6 * len(re.findall(r'const double vre\d+ = fma\(', loop))         # complex product per trie node
    fl += 2 * len(re.findall(r'= fma\(W2_\d+,', loop))                      # W R accumulated
    fl += len(re.findall(r'= (?:imul\()?W2_\d+(?:,| \*)', loop))                # ... its first term, a product
    fl += 2 + 4                                                             # mean and variance sums
    return fl


def tables():
    out = [("order2_bosonic", T.Diagram(W.ORDER2["alpha"], var_is_boson=W.ORDER2["var_is_boson"])),
           ("quadruple_pole", T.Diagram([[1, 0], [1, 0], [1, 0], [1, 0], [1, 1]],
                                        eps=[[1, 0, 0, 0, 0]] * 4 + [[0, 0, 0, 0, 1]], var_is_boson=[0, 1]))]
    for m in (2, 3, 4, 5):
        for i, d in enumerate(T.enumerate_sigma(m)):
            out.append((f"order{m}_{i}", T.Diagram(d["alpha"], eps=d["eps"])))
    return out


def test_model_counts_what_the_generated_forward_computes():
    checked = 0
    for name, D in tables():
        src = D.jit_source("forward")
        info = D.info()
        assert per_sample(src) == info["flops_per_sample"], name
        assert per_frequency(src) == info["flops_per_sample_freq"], name
        checked += 1
    assert checked == 87


def test_shared_prefixes_are_counted_once():
    """The bench's order-4 table: chains of its pole-DAG nodes share prefixes, so some prefix is
    extended by more than one longer prefix (each written once in the generated source)."""
    d = next(x for x in T.enumerate_sigma(4) if x["code"] == tuple(W.ORDER4["code"]))
    src = T.Diagram(d["alpha"], eps=d["eps"]).jit_source("forward")
    parents = re.findall(r'const double pv\d+ = fma\(fv\d+, [^,]+, (pv\d+)\);', src)
    assert max(parents.count(p) for p in set(parents)) >= 2


def signed_prefix_keys(src):
    """Each pole-DAG prefix of a generated kernel as a structural key up to its sign: a chain's
    partial sum and the same steps with every sign flipped are one value (fma(F, -a, -c) =
    -fma(F, a, c) in round-to-nearest), so the generator writes only one of them."""
    canon, keys = {}, []

    def operand(tok):
        tok = tok.strip()
        if tok.startswith("pv") or tok.startswith("-pv"):
            s, c = canon[tok.lstrip("-")]
            return ("node", c), (-s if tok.startswith("-") else s)
        v = float.fromhex(tok)
        return ("leaf", abs(v)), (1 if v > 0 else -1)

    pat = r'const double (pv\d+) = (?:(-?)fv(\d+)|(?:fma|imul_ftz)\(fv(\d+), ([^,)]+)(?:, ([^)]+))?\));'
    for m in re.finditer(pat, src):
        if m.group(3) is not None:                     # +-F: a chain's first step on a unit leaf
            key, sign = ("F", m.group(3)), -1 if m.group(2) else 1
        else:
            (ko, so) = operand(m.group(5))
            add = (m.group(6) or "0.0").strip()        # imul_ftz(F, operand): a first step
            if add == "0.0":
                key, sign = ("first", m.group(4), ko), so
            else:
                sp, cp = canon[add]
                key, sign = ("step", cp, m.group(4), ko, so * sp), sp
        keys.append(key)
        canon[m.group(1)] = (sign, len(keys) - 1 if key not in keys[:-1] else keys.index(key))
    return keys


def test_no_prefix_is_another_with_its_signs_flipped():
    """Every prefix the generated kernels write is distinct up to sign and none multiplies a zero
    coefficient (all 87 tables), and the bench's order-4 table does use flipped prefixes (a negated
    node operand or root)."""
    for name, D in tables():
        src = D.jit_source("forward")
        keys = signed_prefix_keys(src)
        assert len(keys) == len(set(keys)), name
        assert "0x0p+0" not in src, name      # a leaf whose terms cancelled exactly is left out
    d = next(x for x in T.enumerate_sigma(4) if x["code"] == tuple(W.ORDER4["code"]))
    src = T.Diagram(d["alpha"], eps=d["eps"]).jit_source("fused")
    assert re.search(r'fma\(fv\d+, -pv\d+,', src) or re.search(r'W1_\d+ = (?:imul_ftz\()?-pv', src)


# ---- the adjoint: bwd_flops_per_sample counted again from the fused kernel's source

UNIT_LIT = re.compile(r'^-?0x1p\+0$')


def _expr_cost(e, shared):
    """Flops of one generated expression under the model's conventions: fma = 2 (an add where a
    factor is +-1, a product onto 0.0), a product = 1 (free by +-1), an add or subtract = 1,
    negation free.  `shared` holds the group weights' wb * W1 products already counted (the
    compiler forms each once)."""
    e = e.strip()
    while e.startswith("(") and _closing(e, 0) == len(e) - 1:
        e = e[1:-1].strip()
    terms = [t for t in _split_sum(e) if t.strip()]
    if len(terms) > 1:
        return sum(_expr_cost(t, shared) for t in terms) + len(terms) - 1
    if e.startswith("-") and not e.startswith("-0x"):
        return _expr_cost(e[1:], shared)
    m = re.match(r'^(fma|imul_ftz|imul)\((.*)\)$', e)
    if m and _closing(e, len(m.group(1))) == len(e) - 1:
        args = _split(m.group(2))
        sub = sum(_expr_cost(a, shared) for a in args)
        units = sum(bool(UNIT_LIT.match(a.strip())) for a in args[:2])
        if m.group(1) == "fma":
            if args[2].strip() == "0.0":
                return sub + (0 if units else 1)
            return sub + (1 if units else 2)
        return sub + (0 if units else 1)
    factors = _split(e, "*")
    if len(factors) > 1:
        sub = sum(_expr_cost(f, shared) for f in factors)
        names = [f.strip() for f in factors]
        n = sum(1 for f in names[1:] if not UNIT_LIT.match(f))
        if UNIT_LIT.match(names[0]):
            n -= 0 if len(names) == 1 else (1 if n else 0)
        if names[:2] and names[0] == "wb" and names[1].startswith("W1_"):   # wb * W1 once per group
            if names[1] in shared:
                n -= 1
            shared.add(names[1])
        return sub + max(n, 0)
    return 0


def _split_sum(s):
    """Top-level terms of a sum or difference (a leading sign and the exponent signs of hex
    literals do not split)."""
    out, depth, cur = [], 0, ""
    for i, ch in enumerate(s):
        depth += ch == "("
        depth -= ch == ")"
        if (ch in "+-" and depth == 0 and cur.strip() and not re.search(r"0x[0-9a-f.]+p$", cur)
                and cur.strip()[-1] not in "*(,+-"):   # a unary sign after an operator does not split
            out.append(cur)
            cur = ""
        else:
            cur += ch
    return out + [cur]


def _closing(s, i):
    depth = 0
    for j in range(i, len(s)):
        depth += s[j] == "("
        depth -= s[j] == ")"
        if depth == 0 and s[j] == ")":
            return j
    return -1


def _split(s, sep=","):
    out, depth, cur = [], 0, ""
    for ch in s:
        depth += ch == "("
        depth -= ch == ")"
        if ch == sep and depth == 0:
            out.append(cur)
            cur = ""
        else:
            cur += ch
    return out + [cur]


def reverse_sweep(src):
    """Flops of the reverse sweep (from the combination adjoints to the parameter adjoints)."""
    body = src[src.index("for (long long tile"):]
    a = body.index("double xbar0")
    rev = body[a:body.index("if (act) {", a)]
    fl, shared, lits = 0, set(), {}
    for st in re.split(r"[;{}]", rev):
        st = st.strip()
        if not st or st.startswith("__syncthreads"):
            continue
        st = re.sub(r"^(const )?double ", "", st)
        for part in _split(st):                   # declarations may list several names
            m = re.match(r"^(\w+)\s*(\+=|-=|\*=|=)\s*(.*)$", part.strip())
            if not m:
                continue
            rhs = m.group(3).strip()
            if re.match(r"^-?0x[0-9a-f.]+p[+-]\d+$", rhs):   # a name for a literal (a_ext)
                lits[m.group(1)] = rhs
                continue
            for k, v in lits.items():
                rhs = re.sub(r"\b%s\b" % k, v, rhs)
            fl += _expr_cost(rhs, shared) + (0 if m.group(2) == "=" else 1)
    return fl


def test_adjoint_model_counts_what_the_generated_adjoint_computes():
    """bwd_flops_per_sample = the fused kernel's per-sample forward part (as the forward count, with
    the k_ext lines' energies and gradients, cos and sin: 108 each), the loop inputs p W, and the
    reverse sweep, statement by statement; all 87 tables."""
    checked = 0
    for name, D in tables():
        src = D.jit_source("fused")
        body = src[src.index("for (long long tile"):src.index("if (xr_zero) {")]
        fl = per_sample(src) + 108 * len(re.findall(r"\bline_energy_grad\(", body))
        for m in re.finditer(r"const double sg\d+_d2 = ([^;]+);", body):   # second derivatives
            fl += _expr_cost(m.group(1), set())
        for m in re.finditer(r"const double pW\d+ = ([^;]+);", body):
            fl += _expr_cost(m.group(1), set())
        fl += reverse_sweep(src)
        assert fl == D.info()["bwd_flops_per_sample"], name
        checked += 1
    assert checked == 87

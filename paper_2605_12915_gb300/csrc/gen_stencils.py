"""Generate af_stencils.cuh: the exact frozen acoustic operator of every node
family as nodal stencils on the half-cell lattice, in straight-line CUDA.

Derivation (exact, sympy):
  * Appendix D gives, for a wedge Theta and a monomial X^a Y^b of the local data
    (X, Y in cell units about the node K), the 3x3 block C^Theta_ab acting on
    (pi, u, v) at radius r = c_K tau / h with weight r^{a+b}.
  * Each wedge's data is the Q2 Lagrange interpolant of its cell's nine nodes
    (Sec. 2); expanding the Lagrange basis in monomials about K turns the block
    into a stencil over the cell's nodes, one polynomial in r per node.
  * Summing over the wedges of the family (vertex: four quadrants, edge
    midpoints: two half planes, centre: the full disk; Sec. 3.1) gives the node
    stencil on the lattice of half-cell offsets around K.

Every family is symmetric under x -> -x and y -> -y about its node, so each
(output, input) channel's stencil is even or odd in each direction.  The
generated code therefore first forms, per orbit {(+-a, +-b)}, the needed
even/odd combinations of the nodal values and then contracts them with one
coefficient per orbit and power: about a quarter of the multiply-adds of the
plain stencil.  Only powers r^1..r^4 are emitted; the r^0 part is the identity
(the increments are what the step needs).  The ee (even-even) combinations are
taken in deviation form (minus the node's own value), which is exact because
the r^q (q >= 1) coefficients of every even-even channel sum to zero, and keeps
FP32 cancellation small.

Outputs per family: Gp[o][q-1] (input p, unscaled) and Guv[o][q-1] (inputs u, v)
for outputs o = (pi, u, v), so that with pi = p / Z_K:
    dp = sum_q r^q (Gp[0] + Z Guv[0]),
    du = sum_q r^q (Gp[1] / Z + Guv[1]),  dv likewise with o = 2.

Run:  python gen_stencils.py  (writes af_stencils.cuh next to this file).
"""
import os
import sys

import sympy as sp

TH = sp.Symbol("theta", real=True)
X, Y = sp.symbols("X Y", real=True)
HALF = sp.Rational(1, 2)

# node families: wedges as (angle lo, angle hi, position of K inside the cell,
# cell units from the cell's lower-left corner)  (Sec. 3.1)
FAMILIES = {
    "V": [(0, sp.pi / 2, (0, 0)), (sp.pi / 2, sp.pi, (1, 0)),
          (sp.pi, 3 * sp.pi / 2, (1, 1)), (3 * sp.pi / 2, 2 * sp.pi, (0, 1))],
    "EV": [(-sp.pi / 2, sp.pi / 2, (0, HALF)), (sp.pi / 2, 3 * sp.pi / 2, (1, HALF))],
    "EH": [(0, sp.pi, (HALF, 0)), (sp.pi, 2 * sp.pi, (HALF, 1))],
    "C": [(0, 2 * sp.pi, (HALF, HALF))],
}
CH_OUT = ["pi", "u", "v"]
CH_IN = ["p", "u", "v"]
# parity (x, y) of each (out, in) channel stencil: 0 even, 1 odd
PARITY = {("pi", "p"): (0, 0), ("pi", "u"): (1, 0), ("pi", "v"): (0, 1),
          ("u", "p"): (1, 0), ("u", "u"): (0, 0), ("u", "v"): (1, 1),
          ("v", "p"): (0, 1), ("v", "u"): (1, 1), ("v", "v"): (0, 0)}


def mu(m, n, t0, t1):
    return sp.integrate(sp.cos(TH) ** m * sp.sin(TH) ** n, (TH, t0, t1))


def zeta(j):
    return sp.sqrt(sp.pi) * sp.gamma(sp.Rational(j + 1, 2)) / sp.gamma(sp.Rational(j, 2) + 1)


def block(a, b, t0, t1):
    """Appendix D compact monomial block, (pi,u,v) x (pi,u,v)."""
    q = a + b
    chi = 1 if q == 0 else 1 + sp.Rational(1, q)
    g = q + 1 + 3 * chi
    M = mu(a, b, t0, t1) * zeta(q + 1)
    Xm = mu(a + 2, b, t0, t1) * zeta(q + 3)
    Ym = mu(a + 1, b + 1, t0, t1) * zeta(q + 3)
    Zm = mu(a, b + 2, t0, t1) * zeta(q + 3)
    Px = (q + 2) * mu(a + 1, b, t0, t1) * zeta(q + 2)
    Py = (q + 2) * mu(a, b + 1, t0, t1) * zeta(q + 2)
    B = sp.Matrix([[(q + 1) * M, -Px, -Py], [-Px, g * Xm - chi * M, g * Ym],
                   [-Py, g * Ym, g * Zm - chi * M]]) / (4 * sp.pi)
    if q == 0:
        B += sp.Rational(2, 3) * (t1 - t0) / (2 * sp.pi) * sp.diag(0, 1, 1)
    return B.applyfunc(sp.nsimplify).applyfunc(sp.simplify)


def lagrange(nodes, t):
    out = []
    for k, v in enumerate(nodes):
        e = sp.Integer(1)
        for m, w in enumerate(nodes):
            if m != k:
                e *= (t - w) / (v - w)
        out.append(sp.Poly(sp.expand(e), t))
    return out


def family_stencil(wedges):
    """coef[(dx, dy)][(out, in)][q] with (dx, dy) lattice offsets in half cells."""
    coef = {}
    for t0, t1, (ox, oy) in wedges:
        blocks = {(a, b): block(a, b, t0, t1) for a in range(3) for b in range(3)}
        xs = [sp.Integer(0) - ox, HALF - ox, 1 - ox]
        ys = [sp.Integer(0) - oy, HALF - oy, 1 - oy]
        LX, LY = lagrange(xs, X), lagrange(ys, Y)
        for ix in range(3):
            for iy in range(3):
                off = (int(2 * xs[ix]), int(2 * ys[iy]))
                for a in range(3):
                    ca = LX[ix].coeff_monomial(X ** a)
                    if ca == 0:
                        continue
                    for b in range(3):
                        cb = LY[iy].coeff_monomial(Y ** b)
                        if cb == 0:
                            continue
                        q = a + b
                        for oi, o in enumerate(CH_OUT):
                            for ii, i in enumerate(CH_IN):
                                val = ca * cb * blocks[(a, b)][oi, ii]
                                if val == 0:
                                    continue
                                d = coef.setdefault(off, {}).setdefault((o, i), {})
                                d[q] = sp.simplify(d.get(q, 0) + val)
    return coef


def check_and_orbits(coef):
    """Verify the reflection parities and return {rep: {(o,i): {q: value}}} for
    representative offsets (a, b) with a, b >= 0, q >= 1."""
    reps = {}
    for (dx, dy), chans in coef.items():
        for (o, i), byq in chans.items():
            px, py = PARITY[(o, i)]
            for q, val in byq.items():
                if q == 0:
                    continue
                mirror = coef.get((-dx, dy), {}).get((o, i), {}).get(q, 0)
                assert sp.simplify(mirror - (-1) ** px * val) == 0, ("x parity", dx, dy, o, i, q)
                mirror = coef.get((dx, -dy), {}).get((o, i), {}).get(q, 0)
                assert sp.simplify(mirror - (-1) ** py * val) == 0, ("y parity", dx, dy, o, i, q)
                if dx >= 0 and dy >= 0:
                    if (dx, dy) == (0, 0):
                        continue  # the node itself: zero in deviation form
                    if (px and dx == 0) or (py and dy == 0):
                        assert sp.simplify(val) == 0
                        continue
                    reps.setdefault((dx, dy), {}).setdefault((o, i), {})[q] = sp.simplify(val)
    # deviation form of even-even channels: coefficients of q >= 1 sum to zero
    for ch, par in PARITY.items():
        if par != (0, 0):
            continue
        for q in range(1, 5):
            tot = 0
            for off, chans in coef.items():
                tot += chans.get(ch, {}).get(q, 0)
            assert sp.simplify(tot) == 0, ("ee sum", ch, q)
    return reps


def literal(v):
    s = sp.N(v, 21)
    return "T(%s)" % sp.sstr(s, full_prec=False)


def emit_family(name, reps):
    lines = []
    lines.append("// family %s: %d orbit representatives" % (name, len(reps)))
    lines.append("template <typename T, typename Load>")
    lines.append("__device__ __forceinline__ void af_sac_%s(const Load& L, T pK, T uK, T vK,"
                 " T Gp[3][4], T Guv[3][4]) {" % name)
    lines.append("#pragma unroll")
    lines.append("  for (int o = 0; o < 3; ++o)")
    lines.append("#pragma unroll")
    lines.append("    for (int q = 0; q < 4; ++q) { Gp[o][q] = T(0); Guv[o][q] = T(0); }")
    nfma = 0
    nadd = 0
    for (a, b) in sorted(reps):
        chans = reps[(a, b)]
        lines.append("  {  // orbit (+-%d, +-%d) half cells" % (a, b))
        members = sorted({(sx * a, sy * b) for sx in (1, -1) for sy in (1, -1)},
                         key=lambda m: (-m[0], -m[1]))
        for k, (dx, dy) in enumerate(members):
            lines.append("    const auto n%d = L(%d, %d);" % (k, dx, dy))
        combos = {}
        for fi, f in enumerate(CH_IN):
            kval = {"p": "pK", "u": "uK", "v": "vK"}[f]
            need = {PARITY[(o, f)] for o in CH_OUT if (o, f) in chans}
            acc = ".%s" % f
            if len(members) == 4:
                # members ordered (a,b), (a,-b), (-a,b), (-a,-b)
                m = {(a, b): 0, (a, -b): 1, (-a, b): 2, (-a, -b): 3}
                i1, i3, i2, i4 = m[(a, b)], m[(a, -b)], m[(-a, b)], m[(-a, -b)]
                lines.append("    const T s12%s = n%d%s + n%d%s, d12%s = n%d%s - n%d%s;"
                             % (f, i1, acc, i2, acc, f, i1, acc, i2, acc))
                lines.append("    const T s34%s = n%d%s + n%d%s, d34%s = n%d%s - n%d%s;"
                             % (f, i3, acc, i4, acc, f, i3, acc, i4, acc))
                nadd += 4
                if (0, 0) in need:
                    lines.append("    const T ee%s = (s12%s + s34%s) - T(4) * %s;" % (f, f, f, kval))
                    nadd += 2
                if (0, 1) in need:
                    lines.append("    const T eo%s = s12%s - s34%s;" % (f, f, f))
                    nadd += 1
                if (1, 0) in need:
                    lines.append("    const T oe%s = d12%s + d34%s;" % (f, f, f))
                    nadd += 1
                if (1, 1) in need:
                    lines.append("    const T oo%s = d12%s - d34%s;" % (f, f, f))
                    nadd += 1
            else:
                i1, i2 = 0, 1  # (+,+) then its mirror
                if (0, 0) in need:
                    lines.append("    const T ee%s = (n%d%s + n%d%s) - T(2) * %s;"
                                 % (f, i1, acc, i2, acc, kval))
                    nadd += 2
                odd = [pp for pp in need if pp != (0, 0)]
                for pp in odd:
                    nm = {(1, 0): "oe", (0, 1): "eo", (1, 1): "oo"}[pp]
                    lines.append("    const T %s%s = n%d%s - n%d%s;" % (nm, f, i1, acc, i2, acc))
                    nadd += 1
            combos[f] = need
        for oi, o in enumerate(CH_OUT):
            for f in CH_IN:
                if (o, f) not in chans:
                    continue
                nm = {(0, 0): "ee", (1, 0): "oe", (0, 1): "eo", (1, 1): "oo"}[PARITY[(o, f)]]
                dst = "Gp" if f == "p" else "Guv"
                for q in sorted(chans[(o, f)]):
                    val = chans[(o, f)][q]
                    if val == 0:
                        continue
                    lines.append("    %s[%d][%d] = fma(%s, %s%s, %s[%d][%d]);"
                                 % (dst, oi, q - 1, literal(val), nm, f, dst, oi, q - 1))
                    nfma += 1
        lines.append("  }")
    lines.append("}")
    lines.append("")
    return lines, nfma, nadd


def emit_family_adjoint(name, reps):
    """Transpose of emit_family: given the adjoints lGp, lGuv of the outputs,
    scatter the adjoints of the lattice values through S(dx, dy, lp, lu, lv) and
    accumulate those of the node's own values (deviation form) into lpK, luK, lvK.
    A member (dx, dy) with dx > 0 and its mirror (-dx, dy) go out together as
    S.pair(dx, dy, lp, lu, lv, lp', lu', lv') (the mirror's values second), so that
    a scatter can merge targets that neighbouring nodes of a row share.  Where
    the node's own column is even (families V and EV), the members (2, dy),
    (-2, dy) and (0, dy) hit three consecutive nodes of one family and row; they
    go out together as S.triple(dy, right, left, centre), the values of (0, dy)
    held from their orbit's block in function-scope temporaries."""
    lines = []
    lines.append("// family %s, transposed: lattice adjoints from output adjoints" % name)
    lines.append("template <typename T, typename Scatter>")
    lines.append("__device__ __forceinline__ void af_sac_%s_adj(const Scatter& S, const T lGp[3][4],"
                 " const T lGuv[3][4], T& lpK, T& luK, T& lvK) {" % name)
    # rows (dy) whose (0, dy) member joins the (+-2, dy) members in one triple
    even_col = name in ("V", "EV")
    triple_dy = set()
    if even_col:
        for (a, b) in reps:
            if a == 2 and (0, b) in reps:
                triple_dy |= {b, -b}
    for dy in sorted(triple_dy):
        lines.append("  T c0%s[3];  // the values of member (0, %d), held for its triple" % (
            ("m%d" % -dy) if dy < 0 else ("p%d" % dy), dy))
    def cname(dy):
        return "c0" + (("m%d" % -dy) if dy < 0 else ("p%d" % dy))
    for (a, b) in sorted(reps):
        chans = reps[(a, b)]
        lines.append("  {  // orbit (+-%d, +-%d) half cells" % (a, b))
        members = sorted({(sx * a, sy * b) for sx in (1, -1) for sy in (1, -1)},
                         key=lambda m: (-m[0], -m[1]))
        lam = {}
        for f in CH_IN:
            for par in ((0, 0), (1, 0), (0, 1), (1, 1)):
                terms = []
                for oi, o in enumerate(CH_OUT):
                    if (o, f) not in chans or PARITY[(o, f)] != par:
                        continue
                    src = "lGp" if f == "p" else "lGuv"
                    for q in sorted(chans[(o, f)]):
                        val = chans[(o, f)][q]
                        if val == 0:
                            continue
                        terms.append((literal(val), "%s[%d][%d]" % (src, oi, q - 1)))
                if terms:
                    nm = {(0, 0): "ee", (1, 0): "oe", (0, 1): "eo", (1, 1): "oo"}[par] + f
                    expr = "T(0)"
                    for c, v in terms:
                        expr = "fma(%s, %s, %s)" % (c, v, expr)
                    lines.append("    const T l%s = %s;" % (nm, expr))
                    lam[(f, par)] = "l" + nm
        kname = {"p": "lpK", "u": "luK", "v": "lvK"}
        for f in CH_IN:
            if (f, (0, 0)) in lam:
                lines.append("    %s -= T(%d) * %s;" % (kname[f], len(members), lam[(f, (0, 0))]))
        member_vals = {}
        for (dx, dy) in members:
            sx = 1 if dx >= 0 else -1
            sy = 1 if dy >= 0 else -1
            vals = []
            for f in CH_IN:
                expr = []
                for par, nm in lam_items(lam, f):
                    sgn = (sx if par[0] else 1) * (sy if par[1] else 1)
                    if len(members) == 2 and par != (0, 0):
                        # two-member orbits: the one odd combination is n0 - n1
                        sgn = 1 if (dx, dy) == members[0] else -1
                    expr.append(("+" if sgn > 0 else "-") + " " + nm)
                e = " ".join(expr) if expr else "+ T(0)"
                vals.append("T(0) " + e)
            member_vals[(dx, dy)] = vals
        for (dx, dy) in members:
            vals = member_vals[(dx, dy)]
            if dx == 0 and dy in triple_dy:
                for k in range(3):
                    lines.append("    %s[%d] = %s;" % (cname(dy), k, vals[k]))
                continue
            if dx == 2 and dy in triple_dy:
                mv = member_vals[(-dx, dy)]
                lines.append("    S.triple(%d, %s, %s, %s," % (dy, vals[0], vals[1], vals[2]))
                lines.append("             %s, %s, %s," % (mv[0], mv[1], mv[2]))
                lines.append("             %s[0], %s[1], %s[2]);" % (cname(dy), cname(dy), cname(dy)))
                continue
            if dx > 0 and (-dx, dy) in member_vals:
                mv = member_vals[(-dx, dy)]
                lines.append("    S.pair(%d, %d, %s, %s, %s," % (dx, dy, vals[0], vals[1], vals[2]))
                lines.append("           %s, %s, %s);" % (mv[0], mv[1], mv[2]))
            elif dx == 0 or (-dx, dy) not in member_vals:
                lines.append("    S(%d, %d, %s, %s, %s);" % (dx, dy, vals[0], vals[1], vals[2]))
        lines.append("  }")
    lines.append("}")
    lines.append("")
    return lines


def lam_items(lam, f):
    out = []
    for par in ((0, 0), (1, 0), (0, 1), (1, 1)):
        if (f, par) in lam:
            out.append((par, lam[(f, par)]))
    return out


def main(out_path):
    header = [
        "// GENERATED by gen_stencils.py -- do not edit.",
        "// Exact frozen acoustic operator (Sec. 3.1; Appendix D compact monomial block)",
        "// as orbit-compressed nodal stencils on the half-cell lattice around a node.",
        "// L(dx, dy) returns the node values (.p, .u, .v) at lattice offset (dx, dy)",
        "// in half cells; pK, uK, vK are the node's own values.  Accumulates, for",
        "// r^1..r^4, Gp[o][q-1] (input p) and Guv[o][q-1] (inputs u, v), o = (pi,u,v).",
        "#pragma once",
        "",
    ]
    body = []
    stats = []
    for name, wedges in FAMILIES.items():
        coef = family_stencil(wedges)
        reps = check_and_orbits(coef)
        lines, nfma, nadd = emit_family(name, reps)
        body += lines
        body += emit_family_adjoint(name, reps)
        stats.append("//   %-2s: %3d multiply-adds, %3d adds" % (name, nfma, nadd))
    text = "\n".join(header + ["// operation counts per node:"] + stats + [""] + body)
    with open(out_path, "w") as f:
        f.write(text)
    print("\n".join(stats))


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(here, "af_stencils.cuh"))

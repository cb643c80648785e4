"""Generator of the u u~ -> t t~ g g amplitude code (csrc/mf_gen_uux.cuh).

    python -m paper_2211_14056_gb300.gen_uux

arXiv:2211.14056 evaluates autogenerated tree-level matrix elements per event
(Sec. 2, Table 1: pp -> t t~ g g includes the q q~ channels).  For two quark
lines (u u~ and t t~) connected by gluons the colour-ordered one-line
recursion of gen_tables does not apply; this generator works at the level of
Feynman diagrams instead:

* the tree diagrams are enumerated by topology: the light line (v~bar(p2)
  ... u(p1)) and the heavy line (u~bar(p3) ... v(p4)) exchange one gluon (the
  "bridge"); each external gluon sits on the light line, the heavy line or
  the bridge, or both gluons first merge into one.  Different flavours on the
  two lines mean no relative fermion signs.  The four-gluon vertex
  contributes one diagram per colour structure (38 in all).
* every diagram's colour factor (products of T^a = lambda^a / 2 along the
  lines, f^abc at gluon vertices) is evaluated as an explicit SU(3) tensor
  and decomposed onto the 12 basis structures (T^A)_{t u}(T^B)_{u~ t~} and
  (T^A)_{t t~}(T^B)_{u~ u} over the ordered splits (A, B) of the two gluons;
  the coefficients are exact small fractions.  The colour matrix of the basis
  is summed exactly over colours.
* the kinematic part is a memoized program of primitive operations
  (external wavefunctions, slashed vertices, propagators, the vector current
  of a fermion line, the three- and four-gluon Lorentz structures), each
  diagram carrying its factors of i from the vertices and propagators
  (Peskin-Schroeder rules, g factored out).

The emitted device function computes, for one helicity configuration of
(u, u~, t~, g, g) and both top helicities, the 12 colour-basis amplitudes
J_b = sum_d c_bd A_d; |M|^2 = (g^8 / (36 * 2)) (1/D) sum J^dagger (D C) J.
"""
import itertools
import os
from fractions import Fraction

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "mf_gen_uux.cuh")

# external legs: 1 u (in), 2 u~ (in), 3 t (out), 4 t~ (out), 5 g (out), 6 g (out)
GLUONS = (5, 6)


# ---------------------------------------------------------------------------
# SU(3)
def su3():
    l = np.zeros((8, 3, 3), dtype=complex)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    T = l / 2
    f = np.zeros((8, 8, 8))
    for a in range(8):
        for b in range(8):
            comm = T[a] @ T[b] - T[b] @ T[a]
            for c in range(8):
                f[a, b, c] = np.real(-2j * np.trace(comm @ T[c]))
    return T, f


# ---------------------------------------------------------------------------
# momenta: tuples of coefficients over (p1 .. p6); K = momentum into the next vertex
def mom(**kw):
    v = [0, 0, 0, 0, 0, 0]
    for k, c in kw.items():
        v[int(k[1]) - 1] += c
    return tuple(v)


def madd(a, b):
    return tuple(x + y for x, y in zip(a, b))


def mneg(a):
    return tuple(-x for x in a)


K_GLUON = {5: mom(p5=-1), 6: mom(p6=-1)}
K56 = madd(K_GLUON[5], K_GLUON[6])


# ---------------------------------------------------------------------------
# the program: a list of (name, op, args); memoized by (op, args)
class Program:
    def __init__(self):
        self.ops = []
        self.memo = {}
        self.moms = {}

    def momentum(self, m):
        if m not in self.moms:
            self.moms[m] = f"K{len(self.moms)}"
        return self.moms[m]

    def add(self, op, *args):
        key = (op, args)
        if key not in self.memo:
            name = f"w{len(self.ops)}"
            self.ops.append((name, op, args))
            self.memo[key] = name
        return self.memo[key]


EXT = ["U1", "V2", "VTB", "UB3", "E5", "E6"]   # wavefunctions supplied by the kernel


def insertion(prog, item):
    """Vector of an insertion ('g5', 'g6', 'g56') and its momentum into the line."""
    if item == 5:
        return "E5", K_GLUON[5]
    if item == 6:
        return "E6", K_GLUON[6]
    if item == "G":
        w = prog.add("vvv", "E5", prog.momentum(K_GLUON[5]), "E6", prog.momentum(K_GLUON[6]))
        return prog.add("gprop", w, prog.momentum(K56)), K56
    raise ValueError(item)


def light_current(prog, left, right):
    """Vector current of the light line with the bridge slot between the
    insertions `left` (from v~bar(p2) towards the slot) and `right` (from
    u(p1) towards the slot); returns (vector, momentum into the next vertex,
    vertices, propagators)."""
    C, P = "U1", mom(p1=1)
    nv = npr = 0
    for item in right:
        V, K = insertion(prog, item)
        C = prog.add("slash_col", V, C)
        nv += 1
        P = madd(P, K)
        C = prog.add("lprop_col", prog.momentum(P), C)
        npr += 1
    Pin = P
    R, P = "V2", mom(p2=-1)
    for item in left:
        V, K = insertion(prog, item)
        R = prog.add("slash_row", R, V)
        nv += 1
        P = madd(P, mneg(K))
        R = prog.add("lprop_row", R, prog.momentum(P))
        npr += 1
    L = prog.add("vcur", R, C)
    nv += 1
    KB = madd(Pin, mneg(P))
    return L, KB, nv, npr


def heavy_column(prog, items):
    """Column spinor of the heavy line with the insertions (vector names and
    momenta into the line, ordered from u~bar(p3) to v(p4)); the amplitude is
    u~bar(p3) . column.  Returns (column, vertices, propagators)."""
    C, P = "VTB", mom(p4=-1)
    nv = npr = 0
    for k, (V, K) in enumerate(reversed(items)):
        C = prog.add("slash_col", V, C)
        nv += 1
        P = madd(P, K)
        if k < len(items) - 1:
            C = prog.add("hprop_col", prog.momentum(P), C)
            npr += 1
    # -p4 + sum K = p3 up to momentum conservation p1 + p2 = p3 + p4 + p5 + p6
    d = tuple(a - b for a, b in zip(P, mom(p3=1)))
    assert d == (0,) * 6 or d == (1, 1, -1, -1, -1, -1)
    return C, nv, npr


def enumerate_diagrams(prog):
    """Every tree diagram: (column, phase exponent, colour description)."""
    diags = []

    def finish(light_items, bridge, heavy_items):
        # light line: items left..right with "B" the bridge slot
        s = light_items.index("B")
        L, KB, nv, npr = light_current(prog, light_items[:s], list(reversed(light_items[s + 1:])))
        gprops = 0
        B = prog.add("gprop", L, prog.momentum(KB))
        gprops += 1
        nv4 = 0
        cur_K = KB
        for step in bridge:
            if step[0] == "v3":
                V, K = insertion(prog, step[1])
                if step[1] == "G":
                    gprops += 1
                W = prog.add("vvv", B, prog.momentum(cur_K), V, prog.momentum(K))
                cur_K = madd(cur_K, K)
            else:   # ("v4", term)
                W = prog.add(f"v4_{step[1]}", B, "E5", "E6")
                cur_K = madd(cur_K, K56)
                nv4 += 1
            B = prog.add("gprop", W, prog.momentum(cur_K))
            gprops += 1
        hv = []
        for item in heavy_items:
            if item == "B":
                hv.append((B, cur_K))
            else:
                V, K = insertion(prog, item)
                if item == "G":
                    gprops += 1
                hv.append((V, K))
        for item in light_items:
            if item == "G":
                gprops += 1
        C, hnv, hnpr = heavy_column(prog, hv)
        # factors of i (Peskin-Schroeder, g factored out): (+i) per quark-gluon
        # vertex i g gamma^mu t^a, (+i) per quark propagator i(p-slash + m)/den,
        # (-i) per gluon propagator -i g_mu_nu/k^2, 1 per three-gluon vertex
        # g f^abc [..], (-i) per four-gluon vertex -i g^2 [..]
        power = {"-i": gprops + nv4, "+i": nv + hnv + npr + hnpr}
        diags.append(dict(column=C, power=power, light=light_items, bridge=bridge, heavy=heavy_items))

    perms = lambda xs: [list(p) for p in itertools.permutations(xs)]
    # 1, 2: both gluons on one line
    for h in perms(["B", 5, 6]):
        finish(["B"], [], h)
    for l in perms(["B", 5, 6]):
        finish(l, [], ["B"])
    # 3: one gluon on each line
    for x, y in ((5, 6), (6, 5)):
        for l in perms(["B", x]):
            for h in perms(["B", y]):
                finish(l, [], h)
    # 4: one gluon on the bridge, the other on a line
    for x, y in ((5, 6), (6, 5)):
        for l in perms(["B", y]):
            finish(l, [("v3", x)], ["B"])
        for h in perms(["B", y]):
            finish(["B"], [("v3", x)], h)
    # 5: both on the bridge
    for x, y in ((5, 6), (6, 5)):
        finish(["B"], [("v3", x), ("v3", y)], ["B"])
    for t in (1, 2, 3):
        finish(["B"], [("v4", t)], ["B"])
    finish(["B"], [("v3", "G")], ["B"])
    # 6: the merged gluon pair on a line
    for l in perms(["B", "G"]):
        finish(l, [], ["B"])
    for h in perms(["B", "G"]):
        finish(["B"], [], h)
    return diags


# ---------------------------------------------------------------------------
# colour
def colour_tensor(d, T, f):
    """Explicit colour tensor [c1, c2, c3, c4, a5, a6] of a diagram."""
    letters = iter("ghijklmnopqrsvwxyz")
    ext = {"c1": "A", "c2": "C", "c3": "D", "c4": "E", 5: "F", 6: "H"}
    factors, subs = [], []
    bridge_in = next(letters)
    # merged pair label (f^{a5 a6 g})
    gl = None
    if "G" in d["light"] or "G" in d["heavy"] or ("v3", "G") in d["bridge"]:
        gl = next(letters)
        factors.append(f)
        subs.append(ext[5] + ext[6] + gl)

    def label(item, side_bridge):
        if item == "B":
            return side_bridge
        if item == "G":
            return gl
        return ext[item]

    # light line: (T^{x1} .. T^{xk})_{c2 c1}
    row = ext["c2"]
    items = d["light"]
    for k, item in enumerate(items):
        col = ext["c1"] if k == len(items) - 1 else next(letters)
        factors.append(T)
        subs.append(label(item, bridge_in) + row + col)
        row = col
    # bridge
    cur = bridge_in
    for step in d["bridge"]:
        nxt = next(letters)
        if step[0] == "v3":
            x = gl if step[1] == "G" else ext[step[1]]
            factors.append(f)
            subs.append(cur + x + nxt)
        else:
            e = next(letters)
            a, b, c, dd = cur, ext[5], ext[6], nxt
            pairs = {1: (a + b + e, c + dd + e), 2: (a + c + e, b + dd + e), 3: (a + dd + e, b + c + e)}[step[1]]
            factors += [f, f]
            subs += list(pairs)
        cur = nxt
    # heavy line: (T^{z1} .. T^{zk})_{c3 c4}
    row = ext["c3"]
    items = d["heavy"]
    for k, item in enumerate(items):
        col = ext["c4"] if k == len(items) - 1 else next(letters)
        factors.append(T)
        subs.append(label(item, cur) + row + col)
        row = col
    spec = ",".join(subs) + "->" + "".join(ext[k] for k in ("c1", "c2", "c3", "c4", 5, 6))
    return np.einsum(spec, *factors, optimize=True)


def _string(T, seq):
    """(T^{a_1} .. T^{a_k})_{ij} as a tensor [a_1 .. a_k, i, j]."""
    M = np.eye(3, dtype=complex)
    for _ in seq:
        M = np.einsum("...ij,ajk->...aik", M, T) if M.ndim > 2 else np.einsum("ij,ajk->aik", M, T)
    return M


def basis_tensors(T):
    """The 12 colour structures [c1, c2, c3, c4, a5, a6] and their labels."""
    splits = []
    for nA in range(3):
        for A in itertools.permutations(GLUONS, nA):
            B = tuple(g for g in GLUONS if g not in A)
            for Bp in itertools.permutations(B):
                splits.append((A, Bp))
    out, labels = [], []
    I3 = np.eye(3)
    for kind in ("tu", "tt"):
        for A, B in splits:
            def line(seq):
                # tensor [i, j, a5, a6] of (T^seq)_{ij} (identity if seq is empty)
                t = np.zeros((3, 3, 8, 8), dtype=complex)
                for a5 in range(8):
                    for a6 in range(8):
                        M = I3.astype(complex)
                        for g in seq:
                            M = M @ T[a5 if g == 5 else a6]
                        t[:, :, a5, a6] = M
                return t
            LA, LB = line(A), line(B)
            if kind == "tu":
                # (T^A)_{c3 c1} (T^B)_{c2 c4}
                t = np.einsum("DAfh,CEfh->ACDEfh", LA, LB)
            else:
                # (T^A)_{c3 c4} (T^B)_{c2 c1}
                t = np.einsum("DEfh,CAfh->ACDEfh", LA, LB)
            # A and B on disjoint gluons: the product is the correct joint tensor
            # only where each gluon index is used once; the line() tensors are
            # constant in unused gluon indices, which the product respects
            out.append(t)
            labels.append((kind, A, B))
    return out, labels


def decompose(tensors, basis):
    Bm = np.stack([b.ravel() for b in basis], axis=1)
    coefs = []
    for t in tensors:
        c, res, _, _ = np.linalg.lstsq(Bm, t.ravel(), rcond=None)
        assert np.abs(Bm @ c - t.ravel()).max() < 1e-10, "colour tensor outside the basis"
        fr = []
        for x in c:
            qr = Fraction(x.real).limit_denominator(1000)
            qi = Fraction(x.imag).limit_denominator(1000)
            assert abs(float(qr) - x.real) < 1e-10 and abs(float(qi) - x.imag) < 1e-10
            fr.append((qr, qi))
        coefs.append(fr)
    return coefs


def colour_matrix(basis):
    """Exact C_bb' = sum over colours of B_b^* B_b' as (integer matrix, denominator)."""
    n = len(basis)
    C = [[None] * n for _ in range(n)]
    for a in range(n):
        for b in range(n):
            v = np.vdot(basis[a], basis[b])
            assert abs(v.imag) < 1e-9
            q = Fraction(v.real).limit_denominator(10000)
            assert abs(float(q) - v.real) < 1e-9
            C[a][b] = q
    D = 1
    for row in C:
        for x in row:
            D = D * x.denominator // np.gcd(D, x.denominator)
    return [[int(x * D) for x in row] for row in C], int(D)


def colour_matrix_exact():
    """(integer matrix, denominator) of the 12 colour structures."""
    T, _ = su3()
    basis, _ = basis_tensors(T)
    return colour_matrix(basis)


def build():
    T, f = su3()
    prog = Program()
    diags = enumerate_diagrams(prog)
    basis, labels = basis_tensors(T)
    coefs = decompose([colour_tensor(d, T, f) for d in diags], basis)
    M, D = colour_matrix(basis)
    return prog, diags, coefs, labels, M, D


# ---------------------------------------------------------------------------
# emission
def _phase(power):
    """(-i)^a (+i)^b as one of 1, i, -1, -i (re, im)."""
    k = (-power["-i"] + power["+i"]) % 4
    return [(1, 0), (0, 1), (-1, 0), (0, -1)][k]


def render():
    prog, diags, coefs, labels, M, D = build()
    n = len(labels)
    L = ["// GENERATED by paper_2211_14056_gb300/gen_uux.py -- do not edit.",
         "// u u~ -> t t~ g g: tree diagrams, colour decomposition onto 12 structures,",
         "// straight-line code of one helicity configuration (see the generator's docstring).",
         "#pragma once",
         "#include \"mf_uux.cuh\"",
         "namespace mf {",
         f"constexpr int kUuxFlows = {n};",
         f"static constexpr int kUuxColourDen = {D};",
         f"static const int kUuxColourNum[{n * n}] = {{{', '.join(str(x) for row in M for x in row)}}};",
         f"// {len(diags)} diagrams; colour basis: " + "; ".join(f"{k} A={A} B={B}" for k, A, B in labels),
         "template <typename T>",
         "__device__ __forceinline__ void uux_amplitudes(const R4<T> (&p)[6], T mt, T mw, const S4<T>& U1, "
         "const S4<T>& V2, const S4<T>& VTB, const S4<T> (&UB3)[2], const V4<T>& E5, const V4<T>& E6, "
         "cplx<T> (&J)[2][" + str(n) + "]) {"]
    for m, name in prog.moms.items():
        terms = " + ".join(f"T({c}) * p[{i}].v[c]" for i, c in enumerate(m) if c != 0)
        L.append(f"  R4<T> {name};")
        L.append(f"#pragma unroll")
        L.append(f"  for (int c = 0; c < 4; ++c) {name}.v[c] = {terms};")
    for name, op, args in prog.ops:
        if op == "slash_col":
            L.append(f"  const S4<T> {name} = apply(make_slash({args[0]}), {args[1]});")
        elif op == "slash_row":
            L.append(f"  const S4<T> {name} = slash_row({args[0]}, {args[1]});")
        elif op == "lprop_col":
            L.append(f"  const S4<T> {name} = lprop_col({args[0]}, {args[1]});")
        elif op == "lprop_row":
            L.append(f"  const S4<T> {name} = lprop_row({args[0]}, {args[1]});")
        elif op == "hprop_col":
            L.append(f"  const S4<T> {name} = hprop_col({args[0]}, mt, mw, {args[1]});")
        elif op == "vcur":
            L.append(f"  const V4<T> {name} = vcur({args[0]}, {args[1]});")
        elif op == "gprop":
            L.append(f"  const V4<T> {name} = gprop({args[0]}, {args[1]});")
        elif op == "vvv":
            L.append(f"  const V4<T> {name} = vvv({args[0]}, {args[1]}, {args[2]}, {args[3]});")
        elif op.startswith("v4_"):
            L.append(f"  const V4<T> {name} = v4_term<{op[3]}>({args[0]}, {args[1]}, {args[2]});")
        else:
            raise ValueError(op)
    L.append("#pragma unroll")
    L.append("  for (int h = 0; h < 2; ++h)")
    L.append("#pragma unroll")
    L.append(f"    for (int b = 0; b < {n}; ++b) J[h][b] = {{T(0), T(0)}};")
    for di, d in enumerate(diags):
        pr, pi = _phase(d["power"])
        # combined constant: (pr + i pi) * (cr + i ci) per basis element
        nz = []
        for b, (cr, ci) in enumerate(coefs[di]):
            zr, zi = pr * cr - pi * ci, pr * ci + pi * cr
            if zr != 0 or zi != 0:
                nz.append((b, zr, zi))
        if not nz:
            continue
        L.append(f"  // diagram {di}: light {d['light']} bridge {d['bridge']} heavy {d['heavy']}")
        L.append("#pragma unroll")
        L.append("  for (int h = 0; h < 2; ++h) {")
        L.append(f"    const cplx<T> a = rowdot(UB3[h], {d['column']});")
        for b, zr, zi in nz:
            if zi == 0:
                L.append(f"    J[h][{b}] = rfma(T({float(zr)!r}), a, J[h][{b}]);")
            elif zr == 0:
                L.append(f"    J[h][{b}] = rfma(T({float(zi)!r}), times_i(a), J[h][{b}]);")
            else:
                L.append(f"    J[h][{b}] = cfma(cplx<T>{{T({float(zr)!r}), T({float(zi)!r})}}, a, J[h][{b}]);")
        L.append("  }")
    L.append("}")
    # colour form over the n structures (D C integer, upper triangle)
    L.append(f"// J^dagger (D C) J over the {n} colour structures (D = {D})")
    L.append("template <typename T>")
    L.append(f"__device__ __forceinline__ T uux_colour_form(const cplx<T> (&J)[{n}]) {{")
    L.append("  T s = T(0);")
    for a in range(n):
        terms = [(b, Fraction(M[a][b], 2) if a == b else Fraction(M[a][b])) for b in range(a, n) if M[a][b] != 0]
        if not terms:
            continue
        b0, c0 = terms[0]
        L.append(f"  {{ cplx<T> y = T({float(c0)!r}) * J[{b0}];")
        for b, c in terms[1:]:
            L.append(f"    y = rfma(T({float(c)!r}), J[{b}], y);")
        L.append(f"    s = fma(J[{a}].r, y.r, fma(J[{a}].i, y.i, s)); }}")
    L.append("  return T(2) * s;")
    L.append("}")
    L.append("}  // namespace mf")
    return "\n".join(L) + "\n"


def main():
    src = render()
    with open(OUT, "w") as fh:
        fh.write(src)
    print(f"wrote {OUT} ({len(src.splitlines())} lines)")


if __name__ == "__main__":
    main()

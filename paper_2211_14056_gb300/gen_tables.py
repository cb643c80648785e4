"""Build-time generator for the heavy-quark-pair + n-gluon device code.

Writes ``csrc/mf_gen_ttng.cuh``:

* the exact colour matrix of the trace basis c_sigma = (T^{a_sigma1} ... T^{a_sigman})_{ij}
  for n = 2, 3, 4, as integers D*C with the common denominator D.  It is
  computed from the SU(N) completeness relation
      sum_a T^a_{ij} T^a_{kl} = (delta_il delta_kj - delta_ij delta_kl / N) / 2
  applied to C_{sigma tau} = sum_a Tr(T^{a_sigman}...T^{a_sigma1} T^{a_tau1}...T^{a_taun}),
  summing exactly over the fundamental indices (integer arithmetic);
* tables of the colour-ordered gluon sub-currents ("blocks"): every ordered
  tuple of distinct gluons up to reversal, with its splits into two and three
  consecutive parts (three-gluon and four-gluon vertices);
* straight-line device code, per gluon count, for the heavy-quark line of one
  helicity lane: the suffix currents R(S), the colour-ordered amplitudes
  J_sigma for both top helicities, and the colour sum J^dagger (D C) J.

The quark line is (T^{a_sigma1} ... T^{a_sigman})_{i_t j_tbar}: gluon sigma1
sits next to the outgoing top, so with R() = v(tbar) and
    R(S) = -(P-slash + m)/(P^2 - m^2 + i m Gamma) sum_{S = B S'} G(B)-slash R(S'),
    J_sigma = ubar(t) sum_{sigma = B S'} G(B)-slash R(S'),
every factor i and g is folded out of J (a common phase and g^n).

Run ``python -m paper_2211_14056_gb300.gen_tables`` after changing it; a test
checks that the committed header is current.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np

NC = 3
HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "mf_gen_ttng.cuh")


# ---------------------------------------------------------------------------
# exact colour matrix
def colour_matrix_exact(n):
    """(orders, integer matrix D*C, D) for the trace basis of n gluons."""
    orders = list(itertools.permutations(range(n)))
    L = 2 * n
    idx = np.array(list(itertools.product(range(NC), repeat=L)), dtype=np.int64)   # [NC^L, L]
    col = np.roll(idx, -1, axis=1)          # column index of the generator at position m is i_{m+1}
    C = [[None] * len(orders) for _ in orders]
    for s, sig in enumerate(orders):
        for t, tau in enumerate(orders):
            # positions: sigma reversed, then tau
            seq = list(reversed(sig)) + list(tau)
            pos = {}
            for m, a in enumerate(seq):
                pos.setdefault(a, []).append(m)
            prod = np.ones(idx.shape[0], dtype=np.int64)
            for a, (m1, m2) in pos.items():
                # 2 N * sum_a T^a_{i j} T^a_{k l} = N d_il d_kj - d_ij d_kl  (N = 3)
                i, j, k, l = idx[:, m1], col[:, m1], idx[:, m2], col[:, m2]
                prod *= NC * ((i == l) & (k == j)) - ((i == j) & (k == l))
            C[s][t] = Fraction(int(prod.sum()), (2 * NC) ** n)
    D = 1
    for row in C:
        for x in row:
            D = D * x.denominator // math.gcd(D, x.denominator)
    M = [[int(x * D) for x in row] for row in C]
    return orders, M, D


# ---------------------------------------------------------------------------
# blocks (colour-ordered gluon sub-currents)
def blocks(n):
    out = []
    for k in range(1, n + 1):
        for t in itertools.permutations(range(n), k):
            if k == 1 or t[0] < t[-1]:
                out.append(t)
    return out


def block_ref(t, ids):
    """(id, sign) of an ordered tuple: reversal costs (-1)^(len+1)."""
    if t in ids:
        return ids[t], 1
    r = tuple(reversed(t))
    return ids[r], (-1) ** (len(t) + 1)


def mask(t):
    return sum(1 << g for g in t)


def tables(n):
    bl = blocks(n)
    ids = {t: i for i, t in enumerate(bl)}
    off, acc = [], 0
    for t in bl:
        off.append(acc)
        acc += 1 << len(t)
    first = [0] * (n + 2)
    for k in range(1, n + 2):
        first[k] = sum(1 for t in bl if len(t) < k)
    o3 = {}
    o4 = {}
    for t in bl:
        k = len(t)
        if k < 2:
            continue
        row = []
        for m in range(1, k):
            (a, sa), (b, sb) = block_ref(t[:m], ids), block_ref(t[m:], ids)
            row.append((a, sa, b, sb))
        o3.setdefault(k, []).append(row)
        row4 = []
        for a in range(1, k - 1):
            for b in range(a + 1, k):
                refs = [block_ref(x, ids) for x in (t[:a], t[a:b], t[b:])]
                row4.append(tuple(v for r in refs for v in r))
        o4.setdefault(k, []).append(row4)
    return bl, ids, off, acc, first, o3, o4


# ---------------------------------------------------------------------------
# emission
def _pack(i, s):
    return i | (0x80 if s < 0 else 0)


def emit_tables(n, lines):
    bl, ids, off, nstore, first, o3, o4 = tables(n)
    lines.append(f"// ---- {n} gluons: {len(bl)} blocks, {nstore} stored currents ----")
    lines.append(f"template <> struct TTNG<{n}> {{")
    lines.append(f"  static constexpr int NBLK = {len(bl)};")
    lines.append(f"  static constexpr int NSTORE = {nstore};")
    lines.append(f"  static constexpr int NPERM = {math.factorial(n)};")
    lines.append(f"  static constexpr int FIRST[{n + 2}] = {{{', '.join(map(str, first))}}};")
    lines.append("};")
    lines.append(f"static __constant__ uint8_t kBlkMask{n}[{len(bl)}] = {{{', '.join(str(mask(t)) for t in bl)}}};")
    lines.append(f"static __constant__ uint16_t kBlkOff{n}[{len(bl)}] = {{{', '.join(map(str, off))}}};")
    lines.append(f"template <> __device__ __forceinline__ const uint8_t* blk_mask<{n}>() {{ return kBlkMask{n}; }}")
    lines.append(f"template <> __device__ __forceinline__ const uint16_t* blk_off<{n}>() {{ return kBlkOff{n}; }}")
    for k in range(2, n + 1):
        flat3 = []
        for row in o3[k]:
            for (a, sa, b, sb) in row:
                flat3 += [_pack(a, sa), _pack(b, sb)]
        lines.append(f"static __constant__ uint8_t kO3_{n}_{k}[{len(flat3)}] = {{{', '.join(map(str, flat3))}}};")
        lines.append(f"template <> __device__ __forceinline__ const uint8_t* o3_table<{n}, {k}>() {{ return kO3_{n}_{k}; }}")
        if k >= 3:
            flat4 = []
            for row in o4[k]:
                for (a, sa, b, sb, c, sc) in row:
                    flat4 += [_pack(a, sa), _pack(b, sb), _pack(c, sc)]
            lines.append(f"static __constant__ uint8_t kO4_{n}_{k}[{len(flat4)}] = {{{', '.join(map(str, flat4))}}};")
            lines.append(f"template <> __device__ __forceinline__ const uint8_t* o4_table<{n}, {k}>() {{ return kO4_{n}_{k}; }}")


def emit_lane(n, lines, colour):
    """Straight-line quark-line code for one helicity lane."""
    bl, ids, off, nstore, first, o3, o4 = tables(n)
    orders, M, D = colour
    oid = {o: i for i, o in enumerate(orders)}
    L = []
    L.append("// One lane: fixed gluon helicities (word H) and tbar helicity (spinor vb).")
    L.append("// Returns sum over both top helicities of J^dagger (D C) J for the")
    L.append(f"// {math.factorial(n)} colour orderings (integer colour matrix, D = {D}).")
    L.append("template <typename T>")
    L.append(f"__device__ __forceinline__ T lane_colour_sum_{n}(const R4<T>* __restrict__ q, const R4<T>& qtb, T m, T mw,")
    L.append("    const V4<T>* __restrict__ Gs, unsigned H, const S4<T>& vb, const S4<T>& ub0, const S4<T>& ub1,")
    L.append(f"    cplx<T> (&J)[{math.factorial(n)}][2]) {{")

    def need(t):
        """Slash matrix of block t at this lane's helicities, loaded where used."""
        i, s = block_ref(tuple(t), ids)
        msk = mask(bl[i])
        bits = [g for g in range(n) if msk >> g & 1]
        ex = " | ".join(f"(((H >> {g}) & 1u) << {j})" for j, g in enumerate(bits))
        ld = f"Gs[{off[i]} + ({ex})]"
        return f"make_slash({ld})" if s > 0 else f"make_slash(neg({ld}))"

    body = []

    def psum(S):
        terms = " + ".join(f"q[{g}]" for g in S)
        return f"-(qtb + {terms})"

    def rec(suffix, rnames, depth):
        # suffix: tuple of gluons already placed at the tbar end (ordered)
        remaining = [g for g in range(n) if g not in suffix]
        if len(remaining) == 1:
            a = remaining[0]
            sigma = (a,) + suffix
            parts = []
            for l in range(1, n + 1):
                B, Sp = sigma[:l], sigma[l:]
                rn = rnames[Sp] if Sp else "vb"
                parts.append((need(B), rn))
            ind = "  " * depth
            body.append(f"{ind}{{ S4<T> W = apply({parts[0][0]}, {parts[0][1]});")
            for sl, rn in parts[1:]:
                body.append(f"{ind}  apply_acc({sl}, {rn}, W);")
            k = oid[sigma]
            body.append(f"{ind}  J[{k}][0] = rowdot(ub0, W); J[{k}][1] = rowdot(ub1, W); }}")
            return
        for b in remaining:
            S = (b,) + suffix
            name = "R" + "".join(map(str, S))
            ind = "  " * depth
            body.append(f"{ind}{{ S4<T> {name};")
            body.append(f"{ind}  {{ S4<T> X = apply({need(S[:1])}, {rnames[S[1:]] if S[1:] else 'vb'});")
            for l in range(2, len(S) + 1):
                B, Sp = S[:l], S[l:]
                body.append(f"{ind}    apply_acc({need(B)}, {rnames[Sp] if Sp else 'vb'}, X);")
            body.append(f"{ind}    {name} = quark_prop(R4<T>({psum(S)}), m, mw, X); }}")
            rn = dict(rnames)
            rn[S] = name
            rec(S, rn, depth + 1)
            body.append(f"{ind}}}")

    rec((), {}, 1)
    L += body
    # colour sum
    L.append("  T tot = T(0);")
    L.append("#pragma unroll")
    L.append("  for (int h = 0; h < 2; ++h) {")
    L.append("    T s = T(0);")
    P = len(orders)
    for a in range(P):
        terms = []
        for b in range(a, P):
            c = M[a][b]
            if c == 0:
                continue
            coef = Fraction(c, 2) if a == b else Fraction(c)
            terms.append((b, coef))
        if not terms:
            continue
        b0, c0 = terms[0]
        L.append(f"    {{ cplx<T> y = T({float(c0)!r}) * J[{b0}][h];")
        for b, c in terms[1:]:
            L.append(f"      y = rfma(T({float(c)!r}), J[{b}][h], y);")
        L.append(f"      s = fma(J[{a}][h].r, y.r, fma(J[{a}][h].i, y.i, s)); }}")
    L.append("    tot += T(2) * s;")
    L.append("  }")
    L.append("  return tot;")
    L.append("}")
    lines += L


def render():
    lines = [
        "// GENERATED by paper_2211_14056_gb300/gen_tables.py -- do not edit.",
        "// Heavy-quark pair + n gluons: colour matrices, sub-current tables and the",
        "// straight-line quark-line code of one helicity lane (see the generator's",
        "// docstring for the recursion it encodes).",
        "#pragma once",
        "#include \"mf_device.cuh\"",
        "namespace mf {",
        "template <int NG> struct TTNG;",
        "template <int NG, int K> __device__ __forceinline__ const uint8_t* o3_table();",
        "template <int NG, int K> __device__ __forceinline__ const uint8_t* o4_table();",
        "template <int NG> __device__ __forceinline__ const uint8_t* blk_mask();",
        "template <int NG> __device__ __forceinline__ const uint16_t* blk_off();",
        "template <typename T> __device__ __forceinline__ V4<T> neg(const V4<T>& a) {",
        "  V4<T> o;",
        "#pragma unroll",
        "  for (int k = 0; k < 4; ++k) o.c[k] = -a.c[k];",
        "  return o;",
        "}",
    ]
    colours = {}
    for n in (2, 3, 4):
        orders, M, D = colour_matrix_exact(n)
        colours[n] = (orders, M, D)
        P = len(orders)
        flat = [x for row in M for x in row]
        lines.append(f"// colour matrix, {n} gluons: C = M / {D}; orderings lexicographic")
        lines.append(f"static constexpr int kColourDen{n} = {D};")
        lines.append(f"static const int kColourNum{n}[{P * P}] = {{{', '.join(map(str, flat))}}};")
        emit_tables(n, lines)
        emit_lane(n, lines, colours[n])
    lines.append("}  // namespace mf")
    return "\n".join(lines) + "\n"


def main():
    src = render()
    with open(OUT, "w") as f:
        f.write(src)
    print(f"wrote {OUT} ({len(src.splitlines())} lines)")


if __name__ == "__main__":
    main()

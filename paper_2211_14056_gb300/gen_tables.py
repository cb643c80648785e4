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
* the depth-first tree of ordered suffixes of the heavy-quark line (which
  sub-currents build each suffix current R(S) and each amplitude J_sigma), read
  by a loop in the kernel (compact code: every lane of a warp walks the same
  path with its own helicities);
* straight-line code of the colour sum J^dagger (D C) J of one helicity with
  the integer colour matrix as immediates.

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
OUT_ADJ = os.path.join(HERE, "csrc", "mf_gen_adj.cuh")


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
def _pack(i, s, bl, off):
    """16-bit block reference: shared-memory offset of the block's stored
    currents (bits 0-8), its gluon mask (bits 9-12), reversal sign (bit 13)."""
    assert off[i] + (1 << len(bl[i])) <= 512
    return off[i] | (mask(bl[i]) << 9) | ((1 << 13) if s < 0 else 0)


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
                flat3 += [_pack(a, sa, bl, off), _pack(b, sb, bl, off)]
        lines.append(f"static __constant__ uint16_t kO3_{n}_{k}[{len(flat3)}] = {{{', '.join(map(str, flat3))}}};")
        lines.append(f"template <> __device__ __forceinline__ const uint16_t* o3_table<{n}, {k}>() {{ return kO3_{n}_{k}; }}")
        if k >= 3:
            flat4 = []
            for row in o4[k]:
                for (a, sa, b, sb, c, sc) in row:
                    flat4 += [_pack(a, sa, bl, off), _pack(b, sb, bl, off), _pack(c, sc, bl, off)]
            lines.append(f"static __constant__ uint16_t kO4_{n}_{k}[{len(flat4)}] = {{{', '.join(map(str, flat4))}}};")
            lines.append(f"template <> __device__ __forceinline__ const uint16_t* o4_table<{n}, {k}>() {{ return kO4_{n}_{k}; }}")


def lane_paths(n):
    """Depth-first tree of ordered suffixes S (gluons next to the antitop).

    Returns per level l = 1..n-1 a list of entries (suffix, parent index in
    level l-1, block refs of S[:m] for m = 1..l); the entries of one parent are
    contiguous, and level 0 is the empty suffix.  Level n-1 entries also carry
    their completion sigma = (a,) + S: its colour-order index and block refs
    of sigma[:m] for m = 1..n.
    """
    bl, ids, off, nstore, first, o3, o4 = tables(n)
    orders = list(itertools.permutations(range(n)))
    oid = {o: i for i, o in enumerate(orders)}
    levels = [[((), -1, [])]]
    for l in range(1, n):
        cur = []
        for pi, (S, _, _) in enumerate(levels[-1]):
            for g in range(n):
                if g in S:
                    continue
                T = (g,) + S
                refs = [block_ref(T[:m], ids) for m in range(1, l + 1)]
                cur.append((T, pi, refs))
        levels.append(cur)
    final = []
    for (S, _, _) in levels[n - 1]:
        a = [g for g in range(n) if g not in S][0]
        sig = (a,) + S
        final.append((oid[sig], [block_ref(sig[:m], ids) for m in range(1, n + 1)]))
    return levels, final


def emit_lane(n, lines, colour):
    """Path tables of the quark line and the colour sum of one helicity lane."""
    levels, final = lane_paths(n)
    bl, _, off, _, _, _, _ = tables(n)
    orders, M, D = colour
    P = len(orders)
    # per level: first child of every parent, suffix mask, block refs
    child0 = [0] * (n + 1)
    for l in range(1, n):
        rows_mask = [mask(S) for (S, _, _) in levels[l]]
        refs = [_pack(i, sg, bl, off) for (_, _, r) in levels[l] for (i, sg) in r]
        firsts = []
        for pi in range(len(levels[l - 1])):
            firsts.append(next(k for k, e in enumerate(levels[l]) if e[1] == pi))
        # the kernel's shared two-gluon suffixes find a level-2 path's parent as p2 // (n - 1)
        assert firsts == [pi * (n - l + 1) for pi in range(len(levels[l - 1]))]
        lines.append(f"static __constant__ uint8_t kPathMask{n}_{l}[{len(rows_mask)}] = {{{', '.join(map(str, rows_mask))}}};")
        lines.append(f"static __constant__ uint16_t kPathBlk{n}_{l}[{len(refs)}] = {{{', '.join(map(str, refs))}}};")
        lines.append(f"static __constant__ uint8_t kPathFirst{n}_{l}[{len(firsts)}] = {{{', '.join(map(str, firsts))}}};")
    fsig = [o for (o, _) in final]
    frefs = [_pack(i, sg, bl, off) for (_, r) in final for (i, sg) in r]
    if n == 4:
        # level-3 paths (a, b, c) paired by their missing gluon g: for every last
        # gluon c and every g != c, the two paths over {a, b} = rest \ {c, g};
        # lanes that differ only in g's helicity share both currents
        pair, miss = [], []
        for c in range(n):
            for g in range(n):
                if g == c:
                    continue
                two = [k for k, (T, _, _) in enumerate(levels[3]) if T[-1] == c and g not in T]
                assert len(two) == 2
                pair += two
                miss.append(g)
        lines.append(f"static __constant__ uint8_t kL3Pair{n}[{len(pair)}] = {{{', '.join(map(str, pair))}}};")
        lines.append(f"static __constant__ uint8_t kL3Miss{n}[{len(miss)}] = {{{', '.join(map(str, miss))}}};")
    lines.append(f"static __constant__ uint8_t kFinalSigma{n}[{len(fsig)}] = {{{', '.join(map(str, fsig))}}};")
    lines.append(f"static __constant__ uint16_t kFinalBlk{n}[{len(frefs)}] = {{{', '.join(map(str, frefs))}}};")
    lines.append(f"template <> struct Paths<{n}> {{")
    for l in range(1, n):
        lines.append(f"  static __device__ __forceinline__ const uint8_t* mask_{l}() {{ return kPathMask{n}_{l}; }}")
    lines.append("  template <int LV> static __device__ __forceinline__ uint8_t mask(int p) {")
    for l in range(1, n):
        lines.append(f"    if constexpr (LV == {l}) return kPathMask{n}_{l}[p];")
    lines.append("    return 0;")
    lines.append("  }")
    lines.append("  template <int LV> static __device__ __forceinline__ uint16_t blk(int p, int m) {")
    for l in range(1, n):
        lines.append(f"    if constexpr (LV == {l}) return kPathBlk{n}_{l}[p * {l} + m];")
    lines.append("    return 0;")
    lines.append("  }")
    lines.append("  template <int LV> static __device__ __forceinline__ int first(int parent) {")
    for l in range(1, n):
        lines.append(f"    if constexpr (LV == {l}) return kPathFirst{n}_{l}[parent];")
    lines.append("    return 0;")
    lines.append("  }")
    lines.append(f"  static __device__ __forceinline__ uint8_t final_sigma(int p) {{ return kFinalSigma{n}[p]; }}")
    lines.append(f"  static __device__ __forceinline__ uint16_t final_blk(int p, int m) {{ return kFinalBlk{n}[p * {n} + m]; }}")
    lines.append("};")
    # colour sum of one helicity from J held in registers
    L = []
    L.append(f"// J^dagger (D C) J of one helicity over the {P} colour orderings (D = {D}).")
    L.append("template <typename T>")
    L.append(f"__device__ __forceinline__ T colour_form_{n}(const cplx<T> (&J)[{P}]) {{")
    L.append("  T s = T(0);")
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
        L.append(f"  {{ cplx<T> y = T({float(c0)!r}) * J[{b0}];")
        for b, c in terms[1:]:
            L.append(f"    y = rfma(T({float(c)!r}), J[{b}], y);")
        L.append(f"    s = fma(J[{a}].r, y.r, fma(J[{a}].i, y.i, s)); }}")
    L.append("  return T(2) * s;")
    L.append("}")
    L.append(f"template <typename T> __device__ __forceinline__ T colour_form(const cplx<T> (&J)[{P}]) {{ return colour_form_{n}<T>(J); }}")
    lines += L


def colour_orbit_terms(n, colour):
    """The colour form split in two halves of equal code by a symmetry.  The
    relabelling pi of the gluons (0 1)(2 3)... (an involution) maps ordering
    sigma to pi(sigma) and leaves D C invariant (relabelling summed colour
    indices), so the terms c_ab Re(J_a^* J_b) of the form (a <= b) fall into
    orbits {(a, b), (pi a, pi b)}.  Returns (perm, terms): perm[a] = the index
    of pi(sigma_a); terms = [(a, b, c)] with one representative of every orbit
    of two terms at its coefficient and every term its own image (an orbit of
    one) at half its coefficient, so that with J'_a = J_perm[a]
        F(J) + F(J') = J^dagger (D C) J / 2,  F(J) = sum_terms c Re(J_a^* J_b),
    the same straight-line F serving both halves on different data."""
    orders, M, D = colour
    P = len(orders)
    pi = list(range(n))
    for g in range(0, n - 1, 2):
        pi[g], pi[g + 1] = g + 1, g
    perm = [orders.index(tuple(pi[g] for g in o)) for o in orders]
    for a in range(P):
        for b in range(P):
            assert M[perm[a]][perm[b]] == M[a][b]
    seen = set()
    terms = []
    for a in range(P):
        for b in range(a, P):
            if M[a][b] == 0 or (a, b) in seen:
                continue
            c = Fraction(M[a][b], 2) if a == b else Fraction(M[a][b])
            img = tuple(sorted((perm[a], perm[b])))
            seen.add((a, b))
            seen.add(img)
            terms.append((a, b, c if img != (a, b) else c / 2))
    return perm, terms


def emit_colour_orbit(n, lines, colour):
    perm, terms = colour_orbit_terms(n, colour)
    P = len(perm)
    lines.append(f"// Half of J^dagger (D C) J / 2 for {P} orderings by the gluon relabelling")
    lines.append(f"// symmetry (gen_tables.colour_orbit_terms): F(J) + F(J o perm) = J^dagger (D C) J / 2.")
    lines.append(f"static __constant__ uint8_t kColourPerm{n}[{P}] = {{{', '.join(map(str, perm))}}};")
    lines.append("template <typename T>")
    lines.append(f"__device__ __forceinline__ T colour_form_orbit_{n}(const cplx<T> (&J)[{P}]) {{")
    lines.append("  T s = T(0);")
    by_a = {}
    for a, b, c in terms:
        by_a.setdefault(a, []).append((b, c))
    for a in sorted(by_a):
        row = by_a[a]
        b0, c0 = row[0]
        lines.append(f"  {{ cplx<T> y = T({float(c0)!r}) * J[{b0}];")
        for b, c in row[1:]:
            lines.append(f"    y = rfma(T({float(c)!r}), J[{b}], y);")
        lines.append(f"    s = fma(J[{a}].r, y.r, fma(J[{a}].i, y.i, s)); }}")
    lines.append("  return s;")
    lines.append("}")
    lines.append(f"template <typename T> __device__ __forceinline__ T colour_form_orbit(const cplx<T> (&J)[{P}]) "
                 f"{{ return colour_form_orbit_{n}<T>(J); }}")
    lines.append(f"template <> struct ColourPerm<{n}> {{")
    lines.append(f"  static __device__ __forceinline__ int at(int a) {{ return kColourPerm{n}[a]; }}")
    lines.append("};")


def colour_tc_fragments(n, colour):
    """(m-tiles, k-steps, values) of D C as the A operand of mma.m16n8k8 (TF32,
    row-major 16 x 8 tiles), laid out [m-tile][k-step][register][lane]:
    register r of lane l holds row 16 mi + l//4 + 8 (r & 1), column
    8 ks + l % 4 + 4 (r >> 1); rows and columns beyond the orderings are 0.
    The entries are integers of magnitude <= 2048, exact in TF32."""
    orders, M, D = colour
    P = len(orders)
    mt, ks = (P + 15) // 16, (P + 7) // 8
    vals = []
    for mi in range(mt):
        for k in range(ks):
            for r in range(4):
                for lane in range(32):
                    row = 16 * mi + lane // 4 + 8 * (r & 1)
                    col = 8 * k + lane % 4 + 4 * (r >> 1)
                    v = M[row][col] if row < P and col < P else 0
                    assert abs(v) <= 2048
                    vals.append(v)
    return mt, ks, vals


def emit_colour_tc(n, lines, colour):
    mt, ks, vals = colour_tc_fragments(n, colour)
    lines.append(f"// D C as TF32 A fragments of mma.m16n8k8: [m-tile][k-step][register][lane]")
    lines.append(f"template <> struct ColourTC<{n}> {{ static constexpr int MT = {mt}, KS = {ks}; }};")
    lines.append(f"static __device__ const float kColourFragA{n}[{len(vals)}] = "
                 f"{{{', '.join(f'{v}.f' for v in vals)}}};")
    lines.append(f"template <> __device__ __forceinline__ const float* colour_frag_a<{n}>() {{ return kColourFragA{n}; }}")


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
        "template <int NG, int K> __device__ __forceinline__ const uint16_t* o3_table();",
        "template <int NG, int K> __device__ __forceinline__ const uint16_t* o4_table();",
        "template <int NG> __device__ __forceinline__ const uint8_t* blk_mask();",
        "template <int NG> __device__ __forceinline__ const uint16_t* blk_off();",
        "template <int NG> struct Paths;",
        "template <int NG> struct ColourTC;",
        "template <int NG> struct ColourPerm;",
        "template <int NG> __device__ __forceinline__ const float* colour_frag_a();",
        "template <int NG> __device__ __forceinline__ const int* colour_num_dev();",
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
        lines.append(f"static __constant__ int kColourNumD{n}[{P * P}] = {{{', '.join(map(str, flat))}}};")
        lines.append(f"template <> __device__ __forceinline__ const int* colour_num_dev<{n}>() {{ return kColourNumD{n}; }}")
        emit_tables(n, lines)
        emit_lane(n, lines, colours[n])
        emit_colour_tc(n, lines, colours[n])
        emit_colour_orbit(n, lines, colours[n])
    lines.append("}  // namespace mf")
    return "\n".join(lines) + "\n"


def full_block_slots(n):
    """Where the adjoint kernel keeps the adjoints of the n-gluon blocks.

    Each n-gluon block (all gluons, one ordering up to reversal) is used by
    exactly two completions of the quark-line walk, sigma and its reversal.
    Its adjoint is kept in the amplitude rows of the ordering whose completion
    the walk reaches first (those rows are read just before and are dead
    afterwards).  Returns, per completion path p in walk order,
    slot | (block parity << 5) | (first << 7), and per n-gluon block (in
    generator order) its slot."""
    levels, final = lane_paths(n)
    bl, ids, off, nstore, first, o3, o4 = tables(n)
    nfull = first[n + 1] - first[n]
    slot, per_path, uses = {}, [], {}
    for (sig, refs) in final:
        i, _ = refs[n - 1]
        b = i - first[n]
        assert 0 <= b < nfull and len(bl[i]) == n
        uses[b] = uses.get(b, 0) + 1
        is_first = b not in slot
        if is_first:
            slot[b] = sig
        assert slot[b] < 32
        per_path.append(slot[b] | ((b & 1) << 5) | (0x80 if is_first else 0))
    assert sorted(uses) == list(range(nfull)) and set(uses.values()) == {2}
    return per_path, [slot[b] for b in range(nfull)]


def render_adj():
    lines = [
        "// GENERATED by paper_2211_14056_gb300/gen_tables.py -- do not edit.",
        "// Adjoint kernel, four gluons: where the adjoints of the four-gluon",
        "// blocks are kept (the amplitude rows of one of the two colour orderings",
        "// whose completions use the block; see full_block_slots).",
        "#pragma once",
        "#include <cstdint>",
        "namespace mf {",
    ]
    per_path, per_block = full_block_slots(4)
    lines.append("// per completion path (walk order): slot | (block parity << 5) | (first use << 7)")
    lines.append(f"static __constant__ uint8_t kG4Leaf4[{len(per_path)}] = {{{', '.join(map(str, per_path))}}};")
    lines.append("// per four-gluon block (generator order): its slot")
    lines.append(f"static __constant__ uint8_t kG4Slot4[{len(per_block)}] = {{{', '.join(map(str, per_block))}}};")
    lines.append("}  // namespace mf")
    return "\n".join(lines) + "\n"


def main():
    for out, src in ((OUT, render()), (OUT_ADJ, render_adj())):
        with open(out, "w") as f:
            f.write(src)
        print(f"wrote {out} ({len(src.splitlines())} lines)")


if __name__ == "__main__":
    main()

"""Host-side properties of the generated quark-line walk tables (gen_tables).

The four-gluon amplitude kernel shares three-gluon quark currents between
lane pairs: lanes l and l ^ (1 << g) differ only in the helicity of gluon g,
and a current R(S) with g not in S is the same for both.  For every last
gluon c and missing gluon g the table kL3Pair4 lists the two level-3 paths
(a, b, c), (b, a, c); the lane whose g-helicity bit is `bit` computes entry
`bit` and receives entry `bit ^ 1` from its partner.  These tests check, on
the emitted tables, that the exchange is consistent and that every lane ends
up with every level-3 current exactly once, and the depth-first layout the
kernels rely on.
"""
import itertools
import re

from paper_2211_14056_gb300 import gen_tables


def _array(src, name):
    m = re.search(r"%s\[\d+\] = \{([^}]*)\}" % re.escape(name), src)
    return [int(x) for x in m.group(1).split(",")]


def test_level3_pairs_share_their_current():
    src = gen_tables.render()
    pair, miss = _array(src, "kL3Pair4"), _array(src, "kL3Miss4")
    levels, _ = gen_tables.lane_paths(4)
    l3 = [T for (T, _, _) in levels[3]]
    assert len(pair) == 24 and len(miss) == 12
    for c in range(4):
        gs = miss[3 * c:3 * c + 3]
        assert sorted(gs) == sorted(g for g in range(4) if g != c)
        for gi, g in enumerate(gs):
            p0, p1 = pair[(3 * c + gi) * 2], pair[(3 * c + gi) * 2 + 1]
            S0, S1 = l3[p0], l3[p1]
            # both end with c, neither contains g, and they are the two orders of the rest
            assert S0[-1] == c and S1[-1] == c and g not in S0 and g not in S1
            assert S0[:2] == S1[:2][::-1] and set(S0) == set(S1)


def test_every_lane_gets_every_level3_current_once():
    src = gen_tables.render()
    pair, miss = _array(src, "kL3Pair4"), _array(src, "kL3Miss4")
    for H in range(16):
        got = []
        for c in range(4):
            for gi in range(3):
                g = miss[c * 3 + gi]
                bit = (H >> g) & 1
                mine, other = pair[(c * 3 + gi) * 2 + bit], pair[(c * 3 + gi) * 2 + (bit ^ 1)]
                # the partner lane (g's helicity flipped) computes exactly what this lane receives
                partner_bit = ((H ^ (1 << g)) >> g) & 1
                assert pair[(c * 3 + gi) * 2 + partner_bit] == other
                got += [mine, other]
        assert sorted(got) == list(range(24))


def test_depth_first_layout():
    for n in (2, 3, 4):
        levels, final = gen_tables.lane_paths(n)
        for l in range(1, n):
            # children of one parent are contiguous, n - l + 1 of them, in parent order
            parents = [p for (_, p, _) in levels[l]]
            assert parents == sorted(parents)
            assert all(parents.count(p) == n - l + 1 for p in set(parents))
            for (T, p, _) in levels[l]:
                assert T[1:] == levels[l - 1][p][0]
        # the completions are the n! orderings, each once
        assert sorted(o for (o, _) in final) == list(range(len(list(itertools.permutations(range(n))))))


def _first(src, ng):
    m = re.search(r"struct TTNG<%d> \{.*?FIRST\[\d+\] = \{([^}]*)\}" % ng, src, re.S)
    return [int(x) for x in m.group(1).split(",")]


def _hel_blk(ref, first, ng):
    """The helicity-sampled kernels' block index of a reference (mf_hel.cuh,
    hel_blk): stored offsets advance by 2^len per block of length len."""
    off, mask = ref & 511, (ref >> 9) & 15
    length = bin(mask).count("1")
    o0 = sum((first[k + 1] - first[k]) << k for k in range(1, length))
    return first[length] + ((off - o0) >> length)


def test_compact_block_index_inverts_the_stored_offsets():
    """Every reference in the generated tables names, through hel_blk, the
    block whose stored offset and gluon mask it carries."""
    src = gen_tables.render()
    for ng in (2, 3, 4):
        first = _first(src, ng)
        off, msk = _array(src, f"kBlkOff{ng}"), _array(src, f"kBlkMask{ng}")
        assert len(off) == first[ng + 1]
        for b in range(len(off)):
            assert _hel_blk(off[b] | (msk[b] << 9), first, ng) == b
        refs = []
        names = set(re.findall(r"(kO[34]_%d_\d+|kPathBlk%d_\d+|kFinalBlk%d)\[" % (ng, ng, ng), src))
        assert f"kFinalBlk{ng}" in names and f"kO3_{ng}_2" in names and (ng < 3 or f"kO4_{ng}_3" in names)
        for name in names:
            refs += _array(src, name)
        for r in refs:
            b = _hel_blk(r, first, ng)
            assert 0 <= b < len(off) and off[b] == (r & 511) and msk[b] == ((r >> 9) & 15)


def test_walk_block_lengths_follow_their_position():
    """The m-th block reference of a walk path (m = 0, 1, ...) holds m + 1
    gluons, in the node tables (kPathBlk, LV per path) and in the completions
    (kFinalBlk, NG per path): the adjoint kernel takes the block length at
    each of these positions as a compile-time constant (its lane reduction
    over the gluons outside the block is specialised on it)."""
    src = gen_tables.render()
    for ng in (2, 3, 4):
        for lv in range(1, ng):
            refs = _array(src, f"kPathBlk{ng}_{lv}")
            assert len(refs) % lv == 0
            for k, r in enumerate(refs):
                assert bin((r >> 9) & 15).count("1") == k % lv + 1
        refs = _array(src, f"kFinalBlk{ng}")
        assert len(refs) == ng * len(list(itertools.permutations(range(ng))))
        for k, r in enumerate(refs):
            assert bin((r >> 9) & 15).count("1") == k % ng + 1



def test_full_block_adjoint_slots():
    """The adjoint kernel keeps the adjoint of each four-gluon block in the
    amplitude rows of a colour ordering (kG4Leaf4, kG4Slot4): the ordering is
    that of the block's first completion in walk order, both completions of
    the block (sigma and its reversal, the only ones that use it) name it,
    exactly the first is flagged to store, and no two blocks share rows."""
    src = gen_tables.render()
    adj = gen_tables.render_adj()
    leaf, slot = _array(adj, "kG4Leaf4"), _array(adj, "kG4Slot4")
    fsig, fblk = _array(src, "kFinalSigma4"), _array(src, "kFinalBlk4")
    first = _first(src, 4)
    off = _array(src, "kBlkOff4")
    assert len(leaf) == 24 and len(slot) == first[5] - first[4] == 12
    assert len(set(slot)) == 12
    seen = {}
    perms = list(itertools.permutations(range(4)))
    for p in range(24):
        ref = fblk[p * 4 + 3]
        b = next(i for i in range(first[4], first[5]) if off[i] == (ref & 511)) - first[4]
        s, par, is_first = leaf[p] & 31, (leaf[p] >> 5) & 1, bool(leaf[p] & 0x80)
        assert s == slot[b] and par == b & 1
        assert is_first == (b not in seen)
        if is_first:
            assert s == fsig[p]
            seen[b] = p
        else:
            # the second completion is the reversal of the first
            assert perms[fsig[p]] == tuple(reversed(perms[fsig[seen[b]]]))
    assert len(seen) == 12


def test_vertex_split_lengths_follow_their_position():
    """The reversed gluon levels of the adjoint kernel take the length of
    every sub-block of a split as a compile-time constant: the s-th
    three-vertex split of a K-gluon block holds blocks of s + 1 and K - s - 1
    gluons (kO3), the s-th four-vertex split blocks of a, b - a and K - b
    gluons for the s-th pair a < b in generator order (kO4)."""
    src = gen_tables.render()
    pop = lambda r: bin((r >> 9) & 15).count("1")
    for ng in (2, 3, 4):
        for K in range(2, ng + 1):
            o3 = _array(src, f"kO3_{ng}_{K}")
            n3 = K - 1
            assert len(o3) % (2 * n3) == 0
            for blk in range(len(o3) // (2 * n3)):
                for s in range(n3):
                    rl, rr = o3[blk * 2 * n3 + 2 * s], o3[blk * 2 * n3 + 2 * s + 1]
                    assert (pop(rl), pop(rr)) == (s + 1, K - s - 1)
            if K < 3:
                continue
            cuts = [(a, b) for a in range(1, K - 1) for b in range(a + 1, K)]
            o4 = _array(src, f"kO4_{ng}_{K}")
            n4 = len(cuts)
            assert n4 == (K - 1) * (K - 2) // 2 and len(o4) % (3 * n4) == 0
            for blk in range(len(o4) // (3 * n4)):
                for s, (a, b) in enumerate(cuts):
                    r = o4[blk * 3 * n4 + 3 * s:blk * 3 * n4 + 3 * s + 3]
                    assert [pop(x) for x in r] == [a, b - a, K - b]


def test_full_blocks_are_stored_last():
    """The adjoint kernel's sub-current adjoint store holds only the blocks of
    fewer than four gluons (their adjoints land at the blocks' own offsets),
    sized as NSTORE minus the four-gluon blocks' entries: that needs every
    shorter block to lie below the first four-gluon block's offset."""
    src = gen_tables.render()
    first = _first(src, 4)
    off, msk = _array(src, "kBlkOff4"), _array(src, "kBlkMask4")
    nstore = int(re.search(r"struct TTNG<4> \{.*?NSTORE = (\d+);", src, re.S).group(1))
    nfull = first[5] - first[4]
    limit = nstore - (nfull << 4)
    for b in range(len(off)):
        length = bin(msk[b]).count("1")
        if length < 4:
            assert off[b] + (1 << length) <= limit, b
        else:
            assert off[b] >= limit, b
    assert limit == 128

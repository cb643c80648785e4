"""Host-side check of the tensor-core colour sum's data layout.

The CUDA colour sum (MF_FP32_TC) builds the operands of mma.m16n8k8 from the
generated D C fragment table and from the warp's amplitude planes.  This test
replays the kernel's per-lane index arithmetic in numpy, assembles the A, B
and accumulator tiles from the per-lane registers with the fragment layouts of
the PTX ISA (mma.m16n8k8, .tf32), multiplies, scatters the accumulator back to
the lanes and forms the per-event sums.  The result must equal the quadratic
form J^T (D C) J of each event computed directly, so a wrong row, column or
stride anywhere in the layout fails here, without a GPU.
"""
import numpy as np
import pytest

from paper_2211_14056_gb300.gen_tables import colour_matrix_exact, colour_tc_fragments

J_STRIDE = 36


def _a_tile(frag, mi, ks, KS):
    """16 x 8 A tile from the per-lane registers a0..a3."""
    A = np.zeros((16, 8))
    for lane in range(32):
        gid, tig = lane // 4, lane % 4
        for r in range(4):
            A[gid + 8 * (r & 1), tig + 4 * (r >> 1)] = frag[((mi * KS + ks) * 4 + r) * 32 + lane]
    return A


def _emulate(ng, planes):
    orders, M, D = colour_matrix_exact(ng)
    NP = len(orders)
    MT, KS, frag = colour_tc_fragments(ng, (orders, M, D))
    L = 2 << ng
    EPW = 32 // L
    plane = NP * 2 * J_STRIDE
    part = np.zeros((32, EPW))          # per lane, per event of the warp
    for u in range(4):
        P = planes[(u >> 1) * plane:(u >> 1) * plane + plane]
        h = u & 1
        for c in range(4):
            lc0 = 8 * c
            d = np.zeros((MT, 32, 4))
            for ks in range(KS):
                # B fragment registers of every lane
                b = np.zeros((32, 2))
                for lane in range(32):
                    gid, tig = lane // 4, lane % 4
                    s0, s1 = 8 * ks + tig, 8 * ks + tig + 4
                    b[lane, 0] = P[(s0 * 2 + h) * J_STRIDE + lc0 + gid] if s0 < NP else 0.0
                    b[lane, 1] = P[(s1 * 2 + h) * J_STRIDE + lc0 + gid] if s1 < NP else 0.0
                B = np.zeros((8, 8))
                for lane in range(32):
                    gid, tig = lane // 4, lane % 4
                    B[tig, gid] = b[lane, 0]
                    B[tig + 4, gid] = b[lane, 1]
                for mi in range(MT):
                    Y = _a_tile(frag, mi, ks, KS) @ B
                    for lane in range(32):
                        gid, tig = lane // 4, lane % 4
                        for r in range(4):
                            d[mi, lane, r] += Y[gid + 8 * (r >> 1), 2 * tig + (r & 1)]
            for lane in range(32):
                gid, tig = lane // 4, lane % 4
                s = 0.0
                for mi in range(MT):
                    for hf in range(2):
                        sg = 16 * mi + gid + 8 * hf
                        if sg < NP:
                            base = (sg * 2 + h) * J_STRIDE + lc0 + 2 * tig
                            s += d[mi, lane, 2 * hf] * P[base] + d[mi, lane, 2 * hf + 1] * P[base + 1]
                part[lane, lc0 // L] += s
    return part.sum(axis=0)             # the full-warp sum of each event


@pytest.mark.parametrize("ng", [2, 3, 4])
def test_fragment_table_is_the_colour_matrix(ng):
    orders, M, D = colour_matrix_exact(ng)
    NP = len(orders)
    MT, KS, frag = colour_tc_fragments(ng, (orders, M, D))
    full = np.zeros((16 * MT, 8 * KS))
    for mi in range(MT):
        for ks in range(KS):
            full[16 * mi:16 * mi + 16, 8 * ks:8 * ks + 8] = _a_tile(frag, mi, ks, KS)
    np.testing.assert_array_equal(full[:NP, :NP], np.array(M, dtype=float))
    assert not full[NP:, :].any() and not full[:, NP:].any()
    assert max(abs(v) for v in frag) <= 2048


@pytest.mark.parametrize("ng", [2, 3, 4])
def test_emulated_tensor_core_sum_is_the_quadratic_form(ng):
    orders, M, D = colour_matrix_exact(ng)
    NP = len(orders)
    rng = np.random.default_rng(ng)
    planes = rng.normal(size=2 * NP * 2 * J_STRIDE)
    got = _emulate(ng, planes)
    # direct: every lane column n, both top helicities, real and imaginary planes
    C = np.array(M, dtype=float)
    L = 2 << ng
    want = np.zeros(32 // L)
    for pl in range(2):
        P = planes[pl * NP * 2 * J_STRIDE:(pl + 1) * NP * 2 * J_STRIDE].reshape(NP * 2, J_STRIDE)
        for h in range(2):
            B = P[h::2, :32]            # [sigma][lane]
            q = np.einsum("sn,st,tn->n", B, C, B)
            want += q.reshape(32 // L, L).sum(axis=1)
    np.testing.assert_allclose(got, want, rtol=1e-12)


def test_orbit_halves_sum_to_the_colour_form():
    """The two halves of the colour form that the helicity-sampled kernel's
    lanes evaluate (the same straight-line terms on J and on J relabelled by
    the gluon symmetry) add up to J^dagger (D C) J / 2, for random complex J."""
    import numpy as np
    from paper_2211_14056_gb300 import gen_tables
    rng = np.random.default_rng(3)
    for n in (2, 3, 4):
        colour = gen_tables.colour_matrix_exact(n)
        orders, M, D = colour
        perm, terms = gen_tables.colour_orbit_terms(n, colour)
        assert sorted(perm) == list(range(len(orders))) and all(perm[perm[a]] == a for a in range(len(perm)))
        Mf = np.array(M, dtype=float)
        full = 0
        for a in range(len(orders)):
            for b in range(a, len(orders)):
                full += (M[a][b] != 0)
        assert len(terms) <= full // 2 + n * len(orders)      # about half the form's terms per half
        for _ in range(5):
            J = rng.normal(size=len(orders)) + 1j * rng.normal(size=len(orders))

            def F(v):
                return sum(float(c) * np.real(np.conj(v[a]) * v[b]) for a, b, c in terms)

            want = np.real(np.conj(J) @ Mf @ J) / 2
            got = F(J) + F(J[perm])
            assert abs(got - want) <= 1e-12 * np.abs(J).max() ** 2 * np.abs(Mf).sum()

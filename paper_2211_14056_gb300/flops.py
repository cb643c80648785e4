"""Static floating-point operation count of one |M|^2 evaluation.

The roofline of the amplitude kernel is FMA-pipe bound, and its algorithmic
work is the number of real floating-point operations the emitted code performs
per event (an FMA counts 2, a multiply or add 1), derived here from the same
block tables and recursion the generator emits (``gen_tables``), with the
per-primitive counts of ``csrc/mf_device.cuh``:

    complex multiply 6, complex FMA 8, real*complex FMA 4, complex add 2,
    Minkowski product complex.complex 30, real.complex 14, real.real 7,
    slash matrix 8, slash*spinor 56 (accumulating 64), spinor row.column 30,
    quark propagator with its precomputed factor 80, three-gluon vertex 164,
    four-gluon vertex 194 (both including the blocks' reversal sign).

Per event, the mask table (momentum sums, 1/K^2 and the propagator factors,
which depend on no helicity) is built once per gluon subset.

External wavefunctions (square roots, divisions) are counted as 30 each.
"""
import math

from .gen_tables import colour_matrix_exact, tables

CMUL, CFMA, RFMA, CADD = 6, 8, 4, 2
MDOT_VV, MDOT_RV, MDOT_RR = CMUL + 3 * CFMA, 2 + 3 * RFMA, 7
SLASH = 4 * CADD
APPLY, APPLY_ACC = 4 * (CMUL + CFMA), 4 * 2 * CFMA
QPROP = 4 * (CMUL + 2 * RFMA) + 4 * CMUL
ROWDOT = CMUL + 3 * CFMA
O3 = 20 + MDOT_VV + 2 * MDOT_RV + 4 * (RFMA + 2 * CFMA) + 6
O4 = 3 * MDOT_VV + 4 + 4 * 3 * CFMA + 4
EXT = 30


def mask_table_flops(ng):
    """Per-event mask table: for every subset of the gluons the momentum sum,
    P = q_tbar + K, K^2, the propagator denominator (for subsets of outgoing
    gluons also its pair-product form, FP32) and its factor."""
    total = 0
    for m in range(1 << ng):
        k = bin(m).count("1")
        total += 4 * k + 4 + MDOT_RR + (MDOT_RR + 1) + 1 + (2 + 1) + 3
        if m & 3 == 0 and m:
            pairs = k * (k - 1) // 2
            total += pairs * (MDOT_RR + 2) + (MDOT_RR + 2)
    return total


def gluon_current_flops(ng):
    """Shared-memory gluon sub-currents of one event (all helicities)."""
    bl, ids, off, nstore, first, o3, o4 = tables(ng)
    total = 2 * ng * EXT + mask_table_flops(ng)
    for k in range(2, ng + 1):
        nblk = first[k + 1] - first[k]
        items = nblk << k
        n3, n4 = k - 1, (k - 1) * (k - 2) // 2
        # vertices, then the scaling by the tabulated 1/K^2
        per = n3 * O3 + n4 * O4 + 8
        total += items * per
    return total


def shared_suffix_flops(ng):
    """Two-gluon suffix currents, computed once per event by the group: per
    (ordered pair, two helicities, antitop helicity) the v spinor, the level-1
    current and the level-2 current."""
    if ng < 3:
        return 0
    items = ng * (ng - 1) * 8
    return items * (EXT + (SLASH + APPLY + QPROP) + (2 * SLASH + 2 * APPLY + 8 + QPROP))


def lane_flops(ng):
    """Quark line, amplitudes and colour sum of one helicity lane."""
    total = 3 * EXT
    # suffix currents R(S) (the two-gluon ones are shared, see above)
    for l in range(1, ng):
        if l == 2 and ng >= 3:
            continue
        count = math.factorial(ng) // math.factorial(ng - l)
        if ng == 4 and l == 3:
            count //= 2      # shared by the lane pair that differs in the missing gluon's helicity
        total += count * (APPLY + (l - 1) * APPLY_ACC + l * SLASH + 4 * l + QPROP)
    # colour-ordered amplitudes, both top helicities
    total += math.factorial(ng) * (APPLY + (ng - 1) * APPLY_ACC + ng * SLASH + 2 * ROWDOT)
    # colour sum, both top helicities
    orders, M, D = colour_matrix_exact(ng)
    P = len(orders)
    per_h = 0
    for a in range(P):
        terms = [b for b in range(a, P) if M[a][b] != 0]
        if terms:
            per_h += 2 + 4 * (len(terms) - 1) + 4
    total += 2 * (per_h + 2)
    return total


def me2_flops_per_event(ng):
    """Real FP operations of one event's |M|^2 (gluon currents + every lane)."""
    lanes = 2 << ng
    return gluon_current_flops(ng) + shared_suffix_flops(ng) + lanes * (lane_flops(ng) + int(math.log2(lanes)))


def me2_flops_per_event_hel(ng):
    """Real FP operations of |M_h|^2 of one helicity configuration (both top
    helicities), the helicity-sampled kernel's work per event: the mask table,
    one polarisation vector per gluon, one sub-current per block, every suffix
    current and ordered amplitude once, the colour form for each top helicity,
    and the antitop and top spinors."""
    bl, ids, off, nstore, first, o3, o4 = tables(ng)
    total = ng * EXT + mask_table_flops(ng) + 3 * EXT
    for k in range(2, ng + 1):
        nblk = first[k + 1] - first[k]
        n3, n4 = k - 1, (k - 1) * (k - 2) // 2
        total += nblk * (n3 * O3 + n4 * O4 + 8)
    for l in range(1, ng):
        count = math.factorial(ng) // math.factorial(ng - l)
        total += count * (APPLY + (l - 1) * APPLY_ACC + l * SLASH + 4 * l + QPROP)
    total += math.factorial(ng) * (APPLY + (ng - 1) * APPLY_ACC + ng * SLASH + 2 * ROWDOT)
    orders, M, D = colour_matrix_exact(ng)
    P = len(orders)
    per_h = 0
    for a in range(P):
        terms = [b for b in range(a, P) if M[a][b] != 0]
        if terms:
            per_h += 2 + 4 * (len(terms) - 1) + 4
    return total + 2 * (per_h + 2) + 2


def sampler_bytes_per_event(n_final, ndim, pass_fraction, kin_bytes):
    """Algorithmic HBM bytes the sampling kernel (k_sample_rec) writes per
    event: the record (final-state momenta and sqrt(s_hat) in the kinematics
    type, the FP64 weight prefactor, one byte per Vegas bin) plus the 4-byte
    entry of the pass list for the events that pass.  It reads only the Vegas
    edges (shared memory, once per CTA)."""
    return (4 * n_final + 1) * kin_bytes + 8 + ndim + 4 * pass_fraction


if __name__ == "__main__":
    for ng in (2, 3, 4):
        print(ng, gluon_current_flops(ng), lane_flops(ng), me2_flops_per_event(ng), me2_flops_per_event_hel(ng))

"""Static floating-point operation count of one |M|^2 evaluation.

The roofline of the amplitude kernel is FMA-pipe bound, and its algorithmic
work is the number of real floating-point operations the emitted code performs
per event (an FMA counts 2, a multiply or add 1), derived here from the same
block tables and recursion the generator emits (``gen_tables``), with the
per-primitive counts of ``csrc/mf_device.cuh``:

    complex multiply 6, complex FMA 8, real*complex FMA 4, complex add 2,
    Minkowski product complex.complex 30, real.complex 14, real.real 7,
    slash matrix 8, slash*spinor 56 (accumulating 64), spinor row.column 30,
    quark propagator 95, three-gluon vertex 158, four-gluon vertex 188.

External wavefunctions (square roots, divisions) are counted as 30 each.
"""
import math

from .gen_tables import colour_matrix_exact, tables

CMUL, CFMA, RFMA, CADD = 6, 8, 4, 2
MDOT_VV, MDOT_RV, MDOT_RR = CMUL + 3 * CFMA, 2 + 3 * RFMA, 7
SLASH = 4 * CADD
APPLY, APPLY_ACC = 4 * (CMUL + CFMA), 4 * 2 * CFMA
QPROP = 4 * (CMUL + 2 * RFMA) + MDOT_RR + 2 + 3 + 1 + 2 + 4 * CMUL
ROWDOT = CMUL + 3 * CFMA
O3 = 20 + MDOT_VV + 2 * MDOT_RV + 4 * (RFMA + 2 * CFMA)
O4 = 3 * MDOT_VV + 2 + 4 * 3 * CFMA
EXT = 30


def gluon_current_flops(ng):
    """Shared-memory gluon sub-currents of one event (all helicities)."""
    bl, ids, off, nstore, first, o3, o4 = tables(ng)
    total = 2 * ng * EXT
    for k in range(2, ng + 1):
        nblk = first[k + 1] - first[k]
        items = nblk << k
        n3, n4 = k - 1, (k - 1) * (k - 2) // 2
        # each split also sums the momenta of its two sub-blocks (4 adds per gluon)
        per = n3 * (O3 + 4 * k) + n4 * O4 + 4 * k + MDOT_RR + 1 + 8
        total += items * per
    return total


def lane_flops(ng):
    """Quark line, amplitudes and colour sum of one helicity lane."""
    total = 3 * EXT
    # suffix currents R(S)
    for l in range(1, ng):
        count = math.factorial(ng) // math.factorial(ng - l)
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
    return gluon_current_flops(ng) + lanes * (lane_flops(ng) + int(math.log2(lanes)))


if __name__ == "__main__":
    for ng in (2, 3, 4):
        print(ng, gluon_current_flops(ng), lane_flops(ng), me2_flops_per_event(ng))

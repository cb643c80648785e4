"""The roofline's algorithmic work (flops.me2_flops_per_event) against the
structure of the generated tables: the quark-line part recounted by walking
the emitted suffix tree (gen_tables.lane_paths) node by node, and the gluon
part by enumerating every item and split of the block tables."""
import math

import pytest

from paper_2211_14056_gb300 import flops as F
from paper_2211_14056_gb300 import gen_tables


def _walk_flops(n):
    """One lane's quark line: every node of the suffix tree costs its slashed
    products (the first one plain, the others accumulating), the slash
    matrices, the momentum sums of the blocks and the propagator; every
    completion costs its n products and two row products.  Level-2 currents
    come from the shared store (n >= 3); for n = 4 each lane computes half of
    the level-3 currents (the lane-pair exchange)."""
    levels, final = gen_tables.lane_paths(n)
    total = 0
    for l in range(1, n):
        if l == 2 and n >= 3:
            continue
        nodes = len(levels[l])
        if n == 4 and l == 3:
            nodes //= 2
        for (_, _, refs) in levels[l][:nodes]:
            assert len(refs) == l
            total += F.APPLY + (l - 1) * F.APPLY_ACC + l * F.SLASH + 4 * l + F.QPROP
    for (_, refs) in final:
        assert len(refs) == n
        total += F.APPLY + (n - 1) * F.APPLY_ACC + n * F.SLASH + 2 * F.ROWDOT
    return total


@pytest.mark.parametrize("n", [2, 3, 4])
def test_lane_count_follows_the_walk_tables(n):
    orders, M, D = gen_tables.colour_matrix_exact(n)
    P = len(orders)
    per_h = sum(2 + 4 * (len([b for b in range(a, P) if M[a][b] != 0]) - 1) + 4 for a in range(P))
    expect = 3 * F.EXT + _walk_flops(n) + 2 * (per_h + 2)
    assert F.lane_flops(n) == expect


@pytest.mark.parametrize("n", [2, 3, 4])
def test_gluon_count_follows_the_block_tables(n):
    bl, ids, off, nstore, first, o3, o4 = gen_tables.tables(n)
    total = 2 * n * F.EXT + F.mask_table_flops(n)
    for k in range(2, n + 1):
        for b in range(first[k], first[k + 1]):
            splits3 = len(o3[k][b - first[k]])
            splits4 = len(o4[k][b - first[k]]) if k >= 3 else 0
            assert splits3 == k - 1 and splits4 == (k - 1) * (k - 2) // 2
            total += (1 << k) * (splits3 * F.O3 + splits4 * F.O4 + 8)
    assert F.gluon_current_flops(n) == total


def test_event_totals():
    # 2^(n+1) lanes per event, a log2(lanes)-step shuffle sum of the helicities
    for n in (2, 3, 4):
        lanes = 2 << n
        assert F.me2_flops_per_event(n) == (F.gluon_current_flops(n) + F.shared_suffix_flops(n)
                                           + lanes * (F.lane_flops(n) + int(math.log2(lanes))))
    assert [F.me2_flops_per_event(n) for n in (2, 3, 4)] == [7464, 71421, 779316]

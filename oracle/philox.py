"""Philox4x32-10 counter-based generator and the uniform draw used by the path.

Test infrastructure (see ``oracle/__init__``).

Definition: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11, Sec. 4 (Philox): a 4x32-bit counter is passed through ten
rounds of a multiply-hi/lo S-box with a Weyl-sequence key schedule.

The paper under study (arXiv:2211.14056, Sec. 1) draws its random numbers as
whole tensors on the device; the counter-based construction below is what lets
both the CPU and the GPU produce the same stream for any event independently.

Stream layout (both sides implement this independently):
    key     = (seed & 0xffffffff, (seed >> 32) ^ iteration)
    counter = (event & 0xffffffff, event >> 32, dim // 2, 0)
    words (w0, w1, w2, w3) = Philox4x32-10(counter, key)
    dim 2j   uses (w0, w1);  dim 2j+1 uses (w2, w3)
    y = ((w_a << 21) | (w_b >> 11)) * 2**-53      in [0, 1), exact in FP64
A second stream, for decisions taken after the weight (the hit-or-miss
unweighting), uses the same key and counter (event & 0xffffffff, event >> 32,
0, 1): its words (w0, w1) give one uniform per event, independent of the
Vegas uniforms (whose counters end in 0).  A third, for the helicity drawn
per event when helicities are sampled, uses counter (event & 0xffffffff,
event >> 32, 1, 1): the top `bits` bits of its word w0 are the helicity index.
"""
import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF


def _mulhilo(a, b):
    """High and low 32-bit halves of the 64-bit product of two uint32 arrays."""
    p = np.asarray(a, dtype=np.uint64) * np.uint64(b)
    return (p >> np.uint64(32)) & np.uint64(MASK32), p & np.uint64(MASK32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on counters (arrays of uint32 values) with key (k0, k1).

    One round (SC'11, Philox S-box, N=4):
        (hi0, lo0) = mulhilo(M0, c0);  (hi1, lo1) = mulhilo(M1, c2)
        c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
    and the key is bumped by the Weyl constants (W0, W1) between rounds.
    """
    u = lambda x: np.asarray(x, dtype=np.uint64) & np.uint64(MASK32)
    c0, c1, c2, c3 = u(c0), u(c1), u(c2), u(c3)
    k0, k1 = u(k0), u(k1)
    for r in range(10):
        if r > 0:
            k0 = (k0 + np.uint64(W0)) & np.uint64(MASK32)
            k1 = (k1 + np.uint64(W1)) & np.uint64(MASK32)
        hi0, lo0 = _mulhilo(c0, M0)
        hi1, lo1 = _mulhilo(c2, M1)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def words_to_unit(wa, wb):
    """53 random bits -> FP64 in [0, 1): ((wa << 21) | (wb >> 11)) * 2^-53."""
    wa = np.asarray(wa, dtype=np.uint64)
    wb = np.asarray(wb, dtype=np.uint64)
    bits = (wa << np.uint64(21)) | (wb >> np.uint64(11))
    return bits.astype(np.float64) * (2.0 ** -53)


def uniforms(seed, iteration, events, ndim):
    """y[ndim, len(events)]: the FP64 uniforms of the listed global events.

    ``events`` are global event indices (uint64); the result does not depend
    on how events are grouped or sharded.
    """
    ev = np.asarray(events, dtype=np.uint64)
    seed = int(seed)
    k0 = seed & MASK32
    k1 = ((seed >> 32) ^ int(iteration)) & MASK32
    out = np.empty((ndim, ev.size), dtype=np.float64)
    c0 = ev & np.uint64(MASK32)
    c1 = ev >> np.uint64(32)
    for j in range((ndim + 1) // 2):
        w0, w1, w2, w3 = philox4x32_10(c0, c1, np.full_like(ev, j), np.zeros_like(ev), k0, k1)
        out[2 * j] = words_to_unit(w0, w1)
        if 2 * j + 1 < ndim:
            out[2 * j + 1] = words_to_unit(w2, w3)
    return out


def unweight_uniforms(seed, iteration, events):
    """r[len(events)]: the unweighting stream's uniform of each listed event."""
    ev = np.asarray(events, dtype=np.uint64)
    seed = int(seed)
    k0 = seed & MASK32
    k1 = ((seed >> 32) ^ int(iteration)) & MASK32
    w0, w1, _, _ = philox4x32_10(ev & np.uint64(MASK32), ev >> np.uint64(32), np.zeros_like(ev),
                                 np.ones_like(ev), k0, k1)
    return words_to_unit(w0, w1)


def helicity_words(seed, iteration, events):
    """w0[len(events)] (uint64 holding 32 bits): word w0 of counter
    (event_lo, event_hi, 1, 1), the helicity stream's word of each event."""
    ev = np.asarray(events, dtype=np.uint64)
    seed = int(seed)
    k0 = seed & MASK32
    k1 = ((seed >> 32) ^ int(iteration)) & MASK32
    w0, _, _, _ = philox4x32_10(ev & np.uint64(MASK32), ev >> np.uint64(32), np.ones_like(ev),
                                np.ones_like(ev), k0, k1)
    return np.asarray(w0, dtype=np.uint64)


def helicity_draws(seed, iteration, events, bits):
    """h[len(events)]: the helicity index (the top `bits` bits of word w0 of
    counter (event_lo, event_hi, 1, 1)) drawn for each listed event."""
    ev = np.asarray(events, dtype=np.uint64)
    seed = int(seed)
    k0 = seed & MASK32
    k1 = ((seed >> 32) ^ int(iteration)) & MASK32
    w0, _, _, _ = philox4x32_10(ev & np.uint64(MASK32), ev >> np.uint64(32), np.ones_like(ev),
                                np.ones_like(ev), k0, k1)
    return (w0 >> np.uint64(32 - bits)).astype(np.int64)

"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11), written from the published definition. Test infrastructure only.

The paper states no random number generator; the DQMC sweep needs one uniform per flip
attempt and one bit per initial auxiliary field. Reading taken: Philox4x32-10 keyed by
the 64-bit seed (key word 0 = low 32 bits, word 1 = high 32 bits) with a 128-bit counter
(word 0 = l*N + i, word 1 = sweep index, word 2 = chain index, word 3 = tag).

Round (per the SC'11 definition): with multipliers M0, M1 and key (k0, k1),
    (hi0, lo0) = M0 * c0,   (hi1, lo1) = M1 * c2   (full 64-bit products)
    c <- (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)
and the key is bumped by the Weyl constants (W0, W1) between rounds; ten rounds.
"""
import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)

TAG_FLIP = 0
TAG_INIT = 1


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 block function.

    All arguments are integers or integer arrays (broadcast together), each holding a
    32-bit word. Returns the four 32-bit output words as uint64 arrays.
    """
    c0, c1, c2, c3, k0, k1 = (np.asarray(v, dtype=np.uint64) & _MASK
                              for v in (c0, c1, c2, c3, k0, k1))
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    m0 = np.uint64(M0)
    m1 = np.uint64(M1)
    for _ in range(10):
        p0 = m0 * c0          # < 2^64: exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + np.uint64(W0)) & _MASK
        k1 = (k1 + np.uint64(W1)) & _MASK
    return c0, c1, c2, c3


def seed_key(seed):
    """Split a 64-bit seed into the two key words (low word first)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def flip_uniforms(seed, l, N, sweep, chain):
    """Uniforms u = x0 * 2^-32 for the N flip attempts of slice l (0-based) in one sweep.

    u is formed exactly in double: x0 < 2^32 is exact, and the scale is a power of two.
    """
    k0, k1 = seed_key(seed)
    i = np.arange(N, dtype=np.uint64)
    x0, _, _, _ = philox4x32_10(np.uint64(l * N) + i, sweep, chain, TAG_FLIP, k0, k1)
    return x0.astype(np.float64) * 2.0 ** -32


def init_fields(seed, L_tau, N, chain):
    """Initial auxiliary field s(i,l) = -1 if the top bit of x0 is set, else +1.

    Counter (l*N + i, 0, chain, TAG_INIT). Returns int8 array [L_tau][N].
    """
    k0, k1 = seed_key(seed)
    idx = np.arange(L_tau * N, dtype=np.uint64)
    x0, _, _, _ = philox4x32_10(idx, 0, chain, TAG_INIT, k0, k1)
    s = np.where((x0 >> np.uint64(31)) != 0, -1, 1).astype(np.int8)
    return s.reshape(L_tau, N)

"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).

Vectorised over counters with numpy uint64 arithmetic. One call maps a
128-bit counter (c0, c1, c2, c3) and a 64-bit key (k0, k1) to four 32-bit
words. Each of the ten rounds multiplies c0 and c2 by the two Philox
multipliers, mixes the high halves with the other counter words and the
key, and the key is bumped by the two Weyl constants between rounds.
"""

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four output words (uint32 arrays) for the given counters.

    c0..c3 are broadcastable integer arrays (values < 2**32); k0, k1 are
    Python ints (< 2**32).
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    key0 = int(k0) & 0xFFFFFFFF
    key1 = int(k1) & 0xFFFFFFFF
    for _ in range(10):
        p0 = _M0 * c0  # < 2**64, exact in uint64
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        n0 = hi1 ^ c1 ^ np.uint64(key0)
        n1 = lo1
        n2 = hi0 ^ c3 ^ np.uint64(key1)
        n3 = lo0
        c0, c1, c2, c3 = n0, n1, n2, n3
        key0 = (key0 + _W0) & 0xFFFFFFFF
        key1 = (key1 + _W1) & 0xFFFFFFFF
    return (c0.astype(np.uint32), c1.astype(np.uint32),
            c2.astype(np.uint32), c3.astype(np.uint32))


def philox_uniform52(lo_word, hi_word):
    """Map two 32-bit words to a double in the open interval (0, 1).

    u = (floor(w / 2**12) + 0.5) * 2**-52 with w = hi_word * 2**32 + lo_word;
    every value is exact in binary64 and lies in [2**-53, 1 - 2**-53].
    """
    w = (np.asarray(hi_word, dtype=np.uint64) << np.uint64(32)) | np.asarray(lo_word, dtype=np.uint64)
    return ((w >> np.uint64(12)).astype(np.float64) + 0.5) * (2.0 ** -52)

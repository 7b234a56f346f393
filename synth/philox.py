"""Philox4x32-10 counter-based generator (numpy).

Written from the published definition: J. K. Salmon, M. A. Moraes,
R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11 (2011), Sec. 4.2: each round multiplies counter words 0 and 2 by the
two round multipliers, takes the 64-bit products' high and low halves and
mixes them with the odd counter words and the key; the key is bumped by the
two Weyl constants between rounds.  The device twin in synth/csrc/gen.cu
implements the same definition and must agree bit for bit.
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_LO = np.uint64(0xFFFFFFFF)


def philox4x32(c0, c1, c2, c3, k0, k1, rounds=10):
    """Vectorised Philox4x32 over broadcastable uint32 arrays.

    Returns the four output words as uint32 arrays.
    """
    c = [np.asarray(x, dtype=np.uint32) for x in (c0, c1, c2, c3)]
    shape = np.broadcast_shapes(*(x.shape for x in c),
                                np.shape(k0), np.shape(k1))
    c0, c1, c2, c3 = (np.broadcast_to(x, shape).astype(np.uint32) for x in c)
    k0 = np.broadcast_to(np.asarray(k0, dtype=np.uint32), shape).copy()
    k1 = np.broadcast_to(np.asarray(k1, dtype=np.uint32), shape).copy()
    with np.errstate(over="ignore"):
        for _ in range(rounds):
            p0 = c0.astype(np.uint64) * _M0
            p1 = c2.astype(np.uint64) * _M1
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _LO).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _LO).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            k0 = (k0 + _W0).astype(np.uint32)
            k1 = (k1 + _W1).astype(np.uint32)
    return c0, c1, c2, c3


def seed_key(seed):
    """Split a 64-bit seed into the two Philox key words."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.uint32(seed & 0xFFFFFFFF), np.uint32(seed >> 32)

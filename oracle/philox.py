"""Philox4x32-10 counter-based generator (CPU oracle).

Test infrastructure only (see the package docstring).  Written from the published
definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11): ten rounds of two 32x32->64-bit multiplications with the constants
M0 = 0xD2511F53 and M1 = 0xCD9E8D57, the key bumped by the Weyl constants
0x9E3779B9 and 0xBB67AE85 between rounds.  The GPU's training-data generator implements
the same definition on its own; tests compare the two and pin this one to the published
known-answer vectors (tests/golden/philox4x32_10_kat.json).
"""
M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def _round(c, k):
    p0 = M0 * c[0]
    p1 = M1 * c[2]
    hi0, lo0 = p0 >> 32, p0 & MASK
    hi1, lo1 = p1 >> 32, p1 & MASK
    return [hi1 ^ c[1] ^ k[0], lo1, hi0 ^ c[3] ^ k[1], lo0]


def philox4x32_10(counter, key):
    """Four 32-bit outputs for a 4-word counter and a 2-word key."""
    c = [int(v) & MASK for v in counter]
    k = [int(v) & MASK for v in key]
    for r in range(10):
        if r:
            k = [(k[0] + W0) & MASK, (k[1] + W1) & MASK]
        c = _round(c, k)
    return c

"""Philox4x32-10 counter-based generator, written from its published definition
(Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy as 1, 2, 3", SC'11).

TEST INFRASTRUCTURE (part of the oracle; see tracker.py).

One round maps the counter (c0, c1, c2, c3) under key (k0, k1) to
  (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
with the 32x32 -> 64-bit products split into high and low words; the key is bumped
by the Weyl constants (W0, W1) between rounds; ten rounds make Philox4x32-10.

Pinned against an independent implementation of the same generator: cuRAND's host-side
PHILOX4_32_10 generator (run on the CPU through ctypes by the tests) gives, word for word, the
outputs of this function for its counters (block k of the stream for seed s is the output for
counter (k div 65536 in c0:c1, k mod 65536 in c2, 0) and key (lo32 s, hi32 s)). Its parts are
also pinned where mathematics fixes them: the key-schedule increments against their definition
(the golden ratio and sqrt 3 in 32-bit fixed point), the round against its inverse, and the
uniformity of the words.
"""
from __future__ import annotations

MASK32 = 0xFFFFFFFF
M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85


def philox4x32_round(c, k):
    """One Philox-4x32 round (Salmon et al., SC'11): two 32 x 32 -> 64-bit products, their
    high words XORed with the other counter words and the round key, the words permuted."""
    c0, c1, c2, c3 = c
    k0, k1 = k
    p0 = M0 * c0
    p1 = M1 * c2
    return ((p1 >> 32) ^ c1 ^ k0, p1 & MASK32, (p0 >> 32) ^ c3 ^ k1, p0 & MASK32)


def philox4x32_10(ctr, key):
    """Ten rounds; round r uses the key bumped r times."""
    c = tuple(int(v) & MASK32 for v in ctr)
    k0, k1 = int(key[0]) & MASK32, int(key[1]) & MASK32
    for r in range(10):
        c = philox4x32_round(c, (k0, k1))
        k0 = (k0 + W0) & MASK32
        k1 = (k1 + W1) & MASK32
    return c

"""The oracle's Philox4x32-10 against an independent implementation of the same generator:
cuRAND's host-side PHILOX4_32_10 generator (libcurand, which runs on the CPU without a
device), called through ctypes with its legacy ordering (the one cuRAND keeps fixed across
releases). No GPU is needed.

cuRAND's host generator with a 64-bit seed s uses the key (lo32(s), hi32(s)); its pseudo-
random stream is made of 4-word blocks, block k being the output for the counter
(floor(k / 65536) as a 64-bit number in (c0, c1), k mod 65536 in c2, 0 in c3): 65536
subsequences advanced together. A generator offset of 4k words starts the stream at block k.
The tests take that mapping as given and compare every word; a match over thousands of
32-bit words between two separate implementations is no accident, and a changed multiplier,
Weyl constant, round count or word order in the oracle fails it (the last test plants such a
change in the oracle and checks that it does)."""
from __future__ import annotations

import ctypes

import pytest

from oracle import philox

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
CURAND_ORDERING_PSEUDO_LEGACY = 103   # the ordering cuRAND keeps the same across its releases
SUBSEQUENCES = 65536


def _load():
    for name in ("libcurand.so.10", "libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


class HostPhilox:
    def __init__(self, lib, seed):
        self.lib = lib
        self.g = ctypes.c_void_p()
        st = lib.curandCreateGeneratorHost(ctypes.byref(self.g), CURAND_RNG_PSEUDO_PHILOX4_32_10)
        if st != 0:
            pytest.skip(f"curandCreateGeneratorHost returned {st}")
        assert lib.curandSetGeneratorOrdering(self.g, CURAND_ORDERING_PSEUDO_LEGACY) == 0
        assert lib.curandSetPseudoRandomGeneratorSeed(self.g, ctypes.c_ulonglong(seed)) == 0

    def words(self, block, nblocks):
        assert self.lib.curandSetGeneratorOffset(self.g, ctypes.c_ulonglong(4 * block)) == 0
        out = (ctypes.c_uint * (4 * nblocks))()
        assert self.lib.curandGenerate(self.g, out, ctypes.c_size_t(4 * nblocks)) == 0
        return [tuple(out[4 * i:4 * i + 4]) for i in range(nblocks)]

    def close(self):
        self.lib.curandDestroyGenerator(self.g)


@pytest.fixture(scope="module")
def curand():
    lib = _load()
    if lib is None:
        pytest.skip("libcurand is not installed")
    return lib


def counter_of_block(k):
    hi, sub = divmod(k, SUBSEQUENCES)
    return (hi & philox.MASK32, hi >> 32, sub, 0)


def key_of_seed(seed):
    return (seed & philox.MASK32, seed >> 32)


SEEDS = [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 0x00000000DEADBEEF, 0x8000000000000000]


@pytest.mark.parametrize("seed", SEEDS)
def test_first_blocks_match_curand(curand, seed):
    """The first 2048 blocks: subsequences 0..2047 at counter word c2, both key words."""
    gen = HostPhilox(curand, seed)
    got = gen.words(0, 2048)
    gen.close()
    key = key_of_seed(seed)
    for k, w in enumerate(got):
        assert w == philox.philox4x32_10(counter_of_block(k), key), (hex(seed), k)


@pytest.mark.parametrize("block", [SUBSEQUENCES - 1, SUBSEQUENCES, 5 * SUBSEQUENCES + 3,
                                   (1 << 32) * SUBSEQUENCES + 7,            # carry into c1
                                   ((1 << 32) + 0x1234) * SUBSEQUENCES + 0xFFFF,
                                   (0xFFFFFFFF << 32 | 0xFFFFFFFF) // 4 // SUBSEQUENCES * SUBSEQUENCES])
def test_blocks_across_the_counter_words(curand, block):
    """Blocks whose counter reaches c0 and c1 (offsets up to the 64-bit limit of cuRAND)."""
    seed = 0xA5A5A5A55A5A5A5A
    gen = HostPhilox(curand, seed)
    got = gen.words(block, 3)
    gen.close()
    for i, w in enumerate(got):
        assert w == philox.philox4x32_10(counter_of_block(block + i), key_of_seed(seed)), (block, i)


@pytest.mark.parametrize("change", ["M0", "M1", "W0", "W1"])
def test_a_planted_change_in_the_oracle_is_caught(curand, monkeypatch, change):
    """The comparison is sensitive: one flipped bit in a multiplier or a Weyl constant of the
    oracle's Philox breaks the agreement on the first blocks."""
    seed = 0x0123456789ABCDEF
    gen = HostPhilox(curand, seed)
    got = gen.words(0, 4)
    gen.close()
    monkeypatch.setattr(philox, change, getattr(philox, change) ^ 0x10)
    mism = sum(w != philox.philox4x32_10(counter_of_block(k), key_of_seed(seed)) for k, w in enumerate(got))
    assert mism == 4

"""Pin the oracle's Philox4x32-10 to an implementation that is not ours.

cuRAND's host-side generator (CURAND_RNG_PSEUDO_PHILOX4_32_10) runs on the CPU.
With the default ordering, its output word 4*(pos*65536 + sub) + w is word w of
Philox4x32-10(key = seed, counter = (pos_lo, pos_hi, sub, 0)).  The oracle draws
only from counters of that form (c2 < 65536, c3 = 0), so this covers every
counter the method uses.
"""
import ctypes
import os
import random

import numpy as np
import pytest

import oracle

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    cands = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcurand.so"),
             "libcurand.so", "libcurand.so.10"]
    for name in cands:
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("cuRAND host library not available")


def _curand_words(lib, seed, offset, n):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        buf = (ctypes.c_uint32 * n)()
        assert lib.curandGenerate(gen, buf, ctypes.c_size_t(n)) == 0
        return np.frombuffer(buf, dtype=np.uint32).copy()
    finally:
        lib.curandDestroyGenerator(gen)


def test_philox_stream_prefix():
    lib = _curand()
    seed = 0x243F6A8885A308D3
    key = (seed & 0xFFFFFFFF, seed >> 32)
    out = _curand_words(lib, seed, 0, 4 * 65536 * 2)
    rng = random.Random(1)
    for _ in range(400):
        pos, sub = rng.randrange(2), rng.randrange(65536)
        q = 4 * (pos * 65536 + sub)
        assert oracle.philox((pos, 0, sub, 0), key) == [int(x) for x in out[q:q + 4]]


def test_philox_arbitrary_counters_and_keys():
    lib = _curand()
    rng = random.Random(2)
    for _ in range(60):
        seed = rng.getrandbits(64)
        key = (seed & 0xFFFFFFFF, seed >> 32)
        pos = rng.getrandbits(rng.choice([8, 32, 40]))
        sub = rng.randrange(65536)
        q = 4 * (pos * 65536 + sub)
        out = _curand_words(lib, seed, q, 4)
        assert oracle.philox((pos & 0xFFFFFFFF, pos >> 32, sub, 0), key) == [int(x) for x in out]


def test_philox_is_a_function_of_every_counter_word():
    key = (1, 2)
    base = oracle.philox((5, 6, 7, 8), key)
    for w in range(4):
        c = [5, 6, 7, 8]
        c[w] ^= 1
        assert oracle.philox(c, key) != base
    assert oracle.philox((5, 6, 7, 8), (1, 3)) != base

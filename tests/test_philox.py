"""Pins for the oracle's Philox4x32-10 (Salmon et al. 2011): the published
known-answer vectors and, as a library cross-check, cuRAND's host generator."""
import ctypes
import os

import pytest

import oracle as O
from conftest import golden_rows


def test_known_answer_vectors():
    rows = golden_rows("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert O.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def _curand():
    for p in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [1, 7, 0x123456789ABCDEF0])
def test_matches_curand_host_generator(seed):
    L = _curand()
    if L is None:
        pytest.skip("libcurand not available")
    g = ctypes.c_void_p()
    if L.curandCreateGeneratorHost(ctypes.byref(g), 161) != 0:   # CURAND_RNG_PSEUDO_PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        buf = (ctypes.c_uint * 4)()
        assert L.curandGenerate(g, buf, ctypes.c_size_t(4)) == 0
        # first block: counter 0, key = (seed low word, seed high word)
        assert list(buf) == O.philox4x32_10([0, 0, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
    finally:
        L.curandDestroyGenerator(g)

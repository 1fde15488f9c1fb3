"""Pins of the oracle's binary32 integer-deciding arithmetic and its RNG.

Philox4x32-10 is pinned against cuRAND's host-side Philox4_32_10 generator, an
independent implementation of the same published algorithm (Salmon et al.,
SC'11): cuRAND's output block j for seed s equals Philox with counter
{0, 0, j, 0} and key {s lo, s hi}.
"""
import ctypes as C
import ctypes.util
import math
import os

import numpy as np
import pytest


def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand and os.path.exists(cand) if cand.startswith("/") else cand:
            try:
                return C.CDLL(cand)
            except OSError:
                continue
    return None


def _curand_host_blocks(lib, seed, n_words):
    gen = C.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161  # curand.h enum value
    assert lib.curandCreateGeneratorHost(C.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, C.c_ulonglong(seed)) == 0
        buf = np.zeros(n_words, np.uint32)
        assert lib.curandGenerate(gen, buf.ctypes.data_as(C.c_void_p), C.c_size_t(n_words)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return buf.reshape(-1, 4)


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host(oracle_mod, seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    blocks = _curand_host_blocks(lib, seed, 4 * 512)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(512):
        got = oracle_mod.philox4x32_10([0, 0, j, 0], key)
        assert np.array_equal(got, blocks[j]), (seed, j, got, blocks[j])


def test_philox_counter_words_all_matter(oracle_mod):
    key = [7, 9]
    base = oracle_mod.philox4x32_10([1, 2, 3, 4], key)
    for w in range(4):
        ctr = [1, 2, 3, 4]
        ctr[w] ^= 1
        assert not np.array_equal(oracle_mod.philox4x32_10(ctr, key), base)
    assert not np.array_equal(oracle_mod.philox4x32_10([1, 2, 3, 4], [7, 8]), base)


def test_exp2_f32_against_math(oracle_mod):
    # exact at integers, <= 2 ulp elsewhere on the range used (lambda and offsets)
    for n in range(-30, 10):
        assert float(oracle_mod.exp2_f32(float(n))) == 2.0 ** n
    ts = np.linspace(-25.0, 8.0, 4001).astype(np.float32)
    for t in ts:
        got = float(oracle_mod.exp2_f32(float(t)))
        ref = 2.0 ** float(t)
        ulp = float(np.spacing(np.float32(ref)))
        assert abs(got - ref) <= 2 * ulp, (t, got, ref)


def test_kelemen_offsets_log_uniform(oracle_mod):
    """Kelemen's small step: |offset| log-uniform on [sigma s1, sigma s2]."""
    s1, s2 = 1.0 / 1024.0, 1.0 / 64.0
    sigma = np.float32(1.7)
    S2 = np.float32(s2 * 2.0 ** 32)
    sigS2 = float(np.float32(sigma * S2))
    c = float(np.float32(math.log2(s2 / s1)))
    # end points
    assert oracle_mod.kelemen_delta(0, sigS2, c) == int(np.rint(np.float32(sigS2)))
    top = oracle_mod.kelemen_delta(0xFFFFFFFF, sigS2, c)
    assert abs(top - float(sigma) * s1 * 2 ** 32) / (float(sigma) * s1 * 2 ** 32) < 1e-6
    rng = np.random.default_rng(3)
    xs = rng.integers(0, 2 ** 32, 20000, dtype=np.uint64)
    lo, hi = math.log(float(sigma) * s1 * 2 ** 32), math.log(float(sigma) * s2 * 2 ** 32)
    ls = np.array([math.log(oracle_mod.kelemen_delta(int(x), sigS2, c)) for x in xs])
    z = (ls - lo) / (hi - lo)
    assert z.min() > -1e-6 and z.max() < 1 + 1e-6
    # Kolmogorov-Smirnov against U(0,1)
    zs = np.sort(z)
    ks = np.max(np.abs(zs - (np.arange(1, len(zs) + 1) / len(zs))))
    assert ks < 1.63 / math.sqrt(len(zs)) * 1.5

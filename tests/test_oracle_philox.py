"""Pins for the oracle's noise: Philox4x32-10 and the Box-Muller transform.

* Philox is pinned bit-exactly against an independent implementation of
  Philox4x32-10 (Salmon et al., SC'11): cuRAND's host-side generator
  (CURAND_RNG_PSEUDO_PHILOX4_32_10), whose output quad m (for the layout it
  uses) is Philox(counter=((m >> 16) mod 2^32, m >> 48, m & 0xffff, 0),
  key=(seed lo, seed hi)).  That mapping covers both key words, counter
  words 0, 1 and 2 and every round; word 3 is pinned on the GPU against
  cuRAND's device generator (tests/test_gpu_philox_device.py).
* Box-Muller is pinned by distribution tests against the standard normal
  (moments and Kolmogorov-Smirnov) and by its two exact points.
"""
import ctypes
import math
import os

import numpy as np
import pytest

CURAND_PHILOX = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    pytest.skip("libcurand not available")


def _curand_host(seed: int, offset: int, count: int) -> np.ndarray:
    lib = _curand()
    g = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(g), CURAND_PHILOX) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        if offset:
            assert lib.curandSetGeneratorOffset(g, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(count, dtype=np.uint32)
        assert lib.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(count)) == 0
    finally:
        lib.curandDestroyGenerator(g)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 2**64 - 1, 0xDEADBEEF00000000])
def test_philox_matches_curand_host(oracle_lib, seed):
    key = (seed & 0xFFFFFFFF, seed >> 32)
    quads = 300
    ref = _curand_host(seed, 0, 4 * quads)
    for m in range(quads):
        got = oracle_lib.philox4x32_10((m >> 16, 0, m & 0xFFFF, 0), key)
        assert np.array_equal(got, ref[4 * m: 4 * m + 4]), (seed, m)


@pytest.mark.parametrize("quad", [65535, 65536, 65537, 1000 * 65536 + 5, (2**32 - 1) * 65536 + 65535,
                                  2**48 + 5, 3 * 2**48 + 7 * 65536 + 11, 2**61 + 12345])
def test_philox_matches_curand_high_counter_words(oracle_lib, quad):
    """Quads at and beyond 2^48 carry into counter word 1 (m >> 48)."""
    seed = 0x0123456789ABCDEF
    key = (seed & 0xFFFFFFFF, seed >> 32)
    ref = _curand_host(seed, 4 * quad, 4)
    got = oracle_lib.philox4x32_10(((quad >> 16) & 0xFFFFFFFF, quad >> 48, quad & 0xFFFF, 0), key)
    assert np.array_equal(got, ref)


def test_box_muller_exact_points(oracle_lib):
    # u1 = 1 (top word all ones) -> radius 0 -> both normals are exactly 0.
    z0, z1 = oracle_lib.box_muller(0xFFFFFFFF, 0x12345678)
    assert z0 == 0.0 and abs(z1) == 0.0
    # u1 = 1/2, u2 = 1/4 -> radius sqrt(2 ln 2), angle pi/2.
    z0, z1 = oracle_lib.box_muller(((1 << 23) - 1) << 8, (1 << 22) << 8)
    assert abs(z0) < 1e-15
    assert abs(z1 - math.sqrt(2.0 * math.log(2.0))) < 1e-15


def test_noise_is_standard_normal(oracle_lib):
    from scipy import stats
    p = oracle_lib.Params(N=1, seed=7)
    xs = np.array([oracle_lib.noise(p, 0, 3, j, k, e) for j in range(50) for k in range(4) for e in range(400)])
    n = len(xs)
    assert abs(xs.mean()) < 5.0 / math.sqrt(n)
    assert abs(xs.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert abs(stats.kurtosis(xs, fisher=False) - 3.0) < 0.1
    assert stats.kstest(xs, "norm").pvalue > 1e-3
    # the transform's range: radius <= sqrt(-2 ln 2^-24)
    assert np.abs(xs).max() <= math.sqrt(-2.0 * math.log(2.0**-24)) + 1e-12


def test_noise_streams_are_distinct(oracle_lib):
    """Different (iteration, step, sample, robot, tag, seed) give different
    streams: no two of these 200-element blocks agree anywhere."""
    base = oracle_lib.Params(N=1, seed=3, tag=0)
    def block(p, it, i, j, k):
        return np.array([oracle_lib.noise(p, it, i, j, k, e) for e in range(200)])
    ref = block(base, 0, 5, 1, 2)
    others = [block(base, 1, 5, 1, 2), block(base, 0, 6, 1, 2), block(base, 0, 5, 2, 2),
              block(base, 0, 5, 1, 3), block(oracle_lib.Params(N=1, seed=3, tag=1), 0, 5, 1, 2),
              block(oracle_lib.Params(N=1, seed=4, tag=0), 0, 5, 1, 2)]
    for o in others:
        assert not np.any(o == ref)

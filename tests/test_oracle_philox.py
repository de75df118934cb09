"""Pins for the oracle's Philox4x32-10 Rademacher stream (Sec. 2.2 probes).

The paper only asks for i.i.d. Rademacher signs; the stream is fixed as
Philox4x32-10 with key = seed and counter = (i_lo, i_hi, p // 128, 0).  The
oracle's generator is pinned to an external implementation -- cuRAND's host
Philox4_32_10 generator, whose output block t + 65536 r is the Philox block at
counter (r, 0, t, 0) -- and by the statistics a Rademacher stream must have.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest


def _curand():
    cands = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcurand.so"),
             "libcurand.so", "libcurand.so.10", ctypes.util.find_library("curand")]
    for c in cands:
        if not c:
            continue
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def _curand_host_philox(seed: int, count: int) -> np.ndarray:
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161  # enum value in curand.h
    rc = lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10)
    if rc != 0:
        pytest.skip("curandCreateGeneratorHost failed (%d)" % rc)
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(count, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(count)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x1234567890, 0xFFFFFFFF00000001])
def test_philox_blocks_match_curand_host(oracle_mod, seed):
    R = 3
    out = _curand_host_philox(seed, 4 * 65536 * R).reshape(R, 65536, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    rng = np.random.default_rng(seed & 0xFFFF)
    for r in range(R):
        for t in list(range(4)) + list(rng.integers(0, 65536, size=40)):
            got = oracle_mod.philox4x32_10([r, 0, int(t), 0], key)
            np.testing.assert_array_equal(got, out[r, int(t)])


def test_rademacher_bit_mapping_matches_curand(oracle_mod):
    seed = 7
    R = 4  # rows i = 0..3 -> counter word 0; probe blocks p // 128 -> counter word 2
    out = _curand_host_philox(seed, 4 * 65536 * R).reshape(R, 65536, 4)
    for i in range(R):
        for p in [0, 1, 31, 32, 33, 63, 64, 95, 96, 127, 128, 129, 200, 255, 256, 1000]:
            word = out[i, p // 128, (p // 32) % 4]
            bit = (int(word) >> (p % 32)) & 1
            assert oracle_mod.rademacher(seed, R, [p])[i, 0] == (-1.0 if bit else 1.0)


def test_rademacher_statistics(oracle_mod):
    d, M = 200_000, 64
    V = oracle_mod.rademacher(0, d, np.arange(M))
    assert set(np.unique(V)) == {-1.0, 1.0}
    # balanced: mean of d*M signs within 5 sigma of 0
    assert abs(V.mean()) < 5.0 / np.sqrt(d * M)
    # per-probe balance
    assert np.max(np.abs(V.mean(axis=0))) < 5.0 / np.sqrt(d)
    # probes pairwise uncorrelated (Hutchinson needs independent columns)
    C = (V.T @ V) / d
    off = C[~np.eye(M, dtype=bool)]
    assert np.max(np.abs(off)) < 6.0 / np.sqrt(d)
    # neighbouring rows uncorrelated
    assert abs(np.mean(V[1:] * V[:-1])) < 5.0 / np.sqrt((d - 1) * M)
    # different seeds give different streams
    V2 = oracle_mod.rademacher(1, d, np.arange(M))
    assert abs(np.mean(V * V2)) < 5.0 / np.sqrt(d * M)


def test_rademacher_probe_blocks_independent(oracle_mod):
    d = 100_000
    V = oracle_mod.rademacher(3, d, np.array([5, 133, 261]))  # same bit, counter words 0,1,2
    for a in range(3):
        for b in range(a + 1, 3):
            assert abs(np.mean(V[:, a] * V[:, b])) < 5.0 / np.sqrt(d)

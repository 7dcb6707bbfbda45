"""Pins the oracle's Philox4x32-10 (the W = 32 instance of its word-size
generic Philox) to cuRAND's, an independent implementation, on the counters
both streams use: the standalone sampler (counter j, key = seed) and the MLMC
paths (counter (s/4, p, tag) in the upper words)."""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_words():
    import torch
    assert torch.cuda.is_available()
    d = tempfile.mkdtemp(prefix="curand_probe_")
    so = os.path.join(d, "libcurandprobe.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", "-o", so, os.path.join(HERE, "helpers", "curand_philox_words.cu")])
    L = C.CDLL(so)
    L.curand_philox_words.restype = C.c_int
    L.curand_philox_words.argtypes = [C.c_uint64, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]

    def words(seed, lo64, hi64):
        lo = np.array([int(x) for x in lo64], dtype=np.uint64)
        hi = np.array([int(x) for x in hi64], dtype=np.uint64)
        out = np.zeros((lo.size, 4), dtype=np.uint32)
        assert L.curand_philox_words(seed, lo.ctypes.data, hi.ctypes.data, lo.size, out.ctypes.data) == 0
        return out
    return words


def test_standalone_stream_counters(curand_words, orc):
    seeds = [0, 7, 0x1234_5678_9ABC, 2 ** 64 - 1]
    rng = np.random.default_rng(0)
    js = [int(x) for x in range(8)] + [int(x) for x in rng.integers(0, 2 ** 40, 40)]
    js += [2 ** 32 - 1, 2 ** 32, 2 ** 62 + 3, 2 ** 63 + 5, 2 ** 64 - 1]
    for seed in seeds:
        got = curand_words(seed, js, [0] * len(js))
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for j, w in zip(js, got):
            j = int(j)
            ref = orc.philox4([j & 0xFFFFFFFF, j >> 32, 0, 0], key, 32)
            assert [int(x) for x in ref] == [int(x) for x in w], (seed, j)


def test_mlmc_stream_counters(curand_words, orc):
    """Path p, fine step s, tag: counter words (s/4, p mod 2^32, p >> 32, tag)."""
    rng = np.random.default_rng(1)
    cases = [(int(rng.integers(0, 64)), int(rng.integers(0, 2 ** 40)), int(rng.integers(0, 2 ** 32))) for _ in range(40)]
    cases += [(0, 0, 1), (255, 2 ** 32 - 1, 7), (4, 2 ** 33 + 9, 0xFFFFFFFF)]
    seed = 0xDEADBEEF_0BADF00D
    lo = [(s // 4) | ((p & 0xFFFFFFFF) << 32) for s, p, _ in cases]
    hi = [(p >> 32) | (tag << 32) for _, p, tag in cases]
    got = curand_words(seed, lo, hi)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for (s, p, tag), w in zip(cases, got):
        ref = orc.philox4([s // 4, p & 0xFFFFFFFF, p >> 32, tag], key, 32)
        assert [int(x) for x in ref] == [int(x) for x in w], (s, p, tag)

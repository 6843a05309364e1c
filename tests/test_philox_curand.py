"""Philox4x32-10 against an independent implementation: cuRAND's device-API
Philox4_32_10 generator, called (never read) through its public interface.

cuRAND's curand_init(seed, subsequence, offset) starts the counter at
(offset/4 as a 64-bit value in words 0-1, subsequence in words 2-3) with key
(seed_lo, seed_hi); its first curand4 is the Philox block of that counter
when offset is a multiple of 4. The oracle's Philox (pinned by the published
known-answer vectors) must give the same four words for the same counter
and key; the GPU generators equal the oracle bit for bit, so they use the
same function."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle as o

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("curand") / "libcurand_philox.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", os.path.join(HERE, "curand_philox.cu"), "-o", out])
    L = C.CDLL(out)
    L.curand_philox_first.argtypes = [C.c_ulonglong, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    L.curand_philox_first.restype = C.c_int
    return L


def test_oracle_philox_equals_curand(curand_lib):
    rng = np.random.default_rng(4)
    for seed in (0, 1, 0xDEADBEEF, 2**63 + 12345):
        n = 64
        sub = rng.integers(0, 2**63, size=n, dtype=np.uint64)
        sub[:4] = [0, 1, 2**32 - 1, 2**32]
        ctr = rng.integers(0, 2**40, size=n, dtype=np.uint64)
        ctr[:4] = [0, 1, 2**32 - 1, 2**32]
        off = ctr * np.uint64(4)
        out = np.zeros((n, 4), np.uint32)
        assert curand_lib.curand_philox_first(seed, sub.ctypes.data, off.ctypes.data,
                                              out.ctypes.data, n) == 0
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for i in range(n):
            c = [int(ctr[i]) & 0xFFFFFFFF, int(ctr[i]) >> 32,
                 int(sub[i]) & 0xFFFFFFFF, int(sub[i]) >> 32]
            assert o.philox4x32_10(c, key).tolist() == out[i].tolist(), (seed, i)

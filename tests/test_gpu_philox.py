"""The random draw of rule (iii) (Sec. 3) against NVIDIA's implementation:
word 0 of Philox-4x32-10 from the library's step-kernel code
(ts_philox_words) and from the oracle must equal cuRAND's device function
curand_Philox4x32_10 on the same counters and keys."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_cs_0105004_gb300 import transsim as T

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib():
    build = os.path.join(os.path.dirname(HERE), "_build", "tests")  # the in-tree build folder
    os.makedirs(build, exist_ok=True)
    out = os.path.join(build, "libcurand_philox.so")
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                    os.path.join(HERE, "cuda", "curand_philox.cu"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    p = ctypes.POINTER(ctypes.c_uint32)
    L.curand_philox_word0.restype = ctypes.c_int
    L.curand_philox_word0.argtypes = [p, p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, p]
    return L


def _curand(L, c0, c1, seed):
    out = np.zeros(c0.size, np.uint32)
    p = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    rc = L.curand_philox_word0(p(c0), p(c1), seed & 0xFFFFFFFF, seed >> 32, c0.size, p(out))
    assert rc == 0
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x243F6A8885A308D3, 2**64 - 1])
def test_library_and_oracle_draws_equal_curand(curand_lib, seed):
    rng = np.random.default_rng(seed % 1000)
    n = 100_000
    step = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    vid = rng.integers(0, 2**31, n, dtype=np.uint64).astype(np.uint32)
    step[:4] = [0, 1, 0xFFFFFFFF, 10799]
    vid[:4] = [0, 0x7FFFFFFF, 5, 299_999]
    ref = _curand(curand_lib, step, vid, seed)
    lib = T.philox_words(step, vid, seed)
    assert np.array_equal(lib, ref)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(0, n, 9973):
        assert int(oracle.philox4x32_10([step[i], vid[i], 0, 0], key)[0]) == int(ref[i]), i

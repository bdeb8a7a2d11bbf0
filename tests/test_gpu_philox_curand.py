"""Philox4x32-10 pinned to a library routine: curand's device
curand_Philox4x32_10, called in a test kernel, against the oracle's
implementation (written from Salmon et al., SC'11) and the library's
(pbits.philox_fill), on random counters and keys and the published corner
cases."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2007_07379_gb300 import build, pbits

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pbits.load()
    out = str(tmp_path_factory.mktemp("curand") / "libcurand_philox.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", "-o", out, os.path.join(HERE, "curand_philox.cu")])
    lib = ctypes.CDLL(out)
    lib.curand_philox.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
    return lib


def test_three_implementations_agree(curand_lib):
    rng = np.random.default_rng(12)
    n = 4096
    ctr = rng.integers(0, 1 << 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 1 << 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    out = np.zeros((n, 4), dtype=np.uint32)
    rc = curand_lib.curand_philox(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, n)
    assert rc == 0
    for i in range(0, n, 97):
        assert np.array_equal(out[i], oracle.philox4x32_10(ctr[i], key[i])), i
    # the library's device implementation (one key per call)
    for kk in (key[0], key[1], key[5]):
        got = pbits.philox_fill(ctr[:256], (int(kk[0]), int(kk[1])))
        sel = np.ones((256, 2), dtype=np.uint32) * kk
        want = np.zeros((256, 4), dtype=np.uint32)
        rc = curand_lib.curand_philox(np.ascontiguousarray(ctr[:256]).ctypes.data, sel.ctypes.data,
                                      want.ctypes.data, 256)
        assert rc == 0
        assert np.array_equal(got, want)

"""Device primitives against the oracle and against cuRAND's Philox.

exp_ticks: the device integer gap equals the oracle's on every edge of its
definition (both branches of the normalisation, all powers of two +- 16, both
ends of the range) and on random words.  Philox4x32-10: the device generator,
the oracle's and cuRAND's curand_Philox4x32_10 (called, not reimplemented)
agree word for word.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

ac = pytest.importorskip("paper_cs_0502039_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _edge_words():
    rng = np.random.default_rng(1)
    parts = [np.arange(0, 1 << 20, dtype=np.uint64),
             np.arange((1 << 31) - (1 << 19), (1 << 31) + (1 << 19), dtype=np.uint64),
             np.arange((1 << 32) - (1 << 20), 1 << 32, dtype=np.uint64),
             rng.integers(0, 1 << 32, 1 << 22, dtype=np.uint64)]
    pw = [(1 << k) + d for k in range(33) for d in range(-16, 17) if 0 <= (1 << k) + d < (1 << 32)]
    parts.append(np.array(pw, dtype=np.uint64))
    return np.concatenate(parts).astype(np.uint32)


def test_exp_ticks_device_equals_oracle():
    x = _edge_words()
    dx = torch.from_numpy(x.view(np.int32)).cuda()
    out = torch.empty(x.size, dtype=torch.int64, device="cuda")
    ac.ac_dev_exp_ticks(dx.data_ptr(), out.data_ptr(), x.size)
    got = out.cpu().numpy().view(np.uint64)
    ref = oracle.exp_ticks_many(x)
    bad = np.flatnonzero(got != ref)
    assert bad.size == 0, (bad[:10], x[bad[:10]], got[bad[:10]], ref[bad[:10]])


def _curand_lib(tmpdir):
    src = os.path.join(os.path.dirname(__file__), "cuda", "curand_philox_ref.cu")
    so = os.path.join(tmpdir, "libcurandref.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                    "-Xcompiler", "-fPIC", src, "-o", so], check=True)
    lib = ctypes.CDLL(so)
    lib.curand_ref_philox.argtypes = [ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                                      ctypes.c_void_p, ctypes.c_int64]
    lib.curand_ref_philox.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("seed,w2", [(1, 0), (7, 1), (0x5EED0502039, 0), (2**64 - 1, 0), (0, 1)])
def test_philox_device_oracle_and_curand_agree(seed, w2, tmp_path):
    rng = np.random.default_rng(seed % 997)
    n = 1 << 16
    c = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    k = rng.integers(0, 64, n, dtype=np.uint64).astype(np.uint32)
    c[:4] = [0, 1, 2**32 - 1, 4095]
    k[:4] = [0, 1, 2**32 - 1, 0]
    dc = torch.from_numpy(c.view(np.int32)).cuda()
    dk = torch.from_numpy(k.view(np.int32)).cuda()
    out = torch.empty(4 * n, dtype=torch.int32, device="cuda")
    ac.ac_dev_philox(seed, dc.data_ptr(), dk.data_ptr(), w2, out.data_ptr(), n)
    dev = out.cpu().numpy().view(np.uint32).reshape(n, 4)
    ref = oracle.philox_blocks(seed, c, k, w2)
    assert np.array_equal(dev, ref)
    lib = _curand_lib(str(tmp_path))
    out2 = torch.empty(4 * n, dtype=torch.int32, device="cuda")
    assert lib.curand_ref_philox(seed & (2**64 - 1), dc.data_ptr(), dk.data_ptr(), w2, out2.data_ptr(), n) == 0
    cur = out2.cpu().numpy().view(np.uint32).reshape(n, 4)
    assert np.array_equal(cur, ref)

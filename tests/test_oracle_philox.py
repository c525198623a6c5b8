"""Pin the oracle's Philox4x32-10 to an independent implementation.

The counter-based generator is Philox4x32-10 of Salmon, Moraes, Dror and Shaw
(SC'11); the paper only asks for one reproducible pseudo-random sequence per
processing element (Sec. 5), refined here to one counter stream per cell.
triton's ``tl.random.philox`` implements the same published generator; run in
its CPU interpreter it gives reference words for arbitrary counters and keys.
"""
import os

import numpy as np
import pytest

import oracle


def _triton_philox(seed, c0, c1, c2, c3):
    os.environ["TRITON_INTERPRET"] = "1"
    torch = pytest.importorskip("torch")
    triton = pytest.importorskip("triton")
    import triton.language as tl

    @triton.jit
    def kern(o0, o1, o2, o3, a0, a1, a2, a3, seed, N: tl.constexpr):
        i = tl.arange(0, N)
        x0 = tl.load(a0 + i).to(tl.uint32, bitcast=True)
        x1 = tl.load(a1 + i).to(tl.uint32, bitcast=True)
        x2 = tl.load(a2 + i).to(tl.uint32, bitcast=True)
        x3 = tl.load(a3 + i).to(tl.uint32, bitcast=True)
        r0, r1, r2, r3 = tl.random.philox(seed, x0, x1, x2, x3, 10)
        tl.store(o0 + i, r0.to(tl.int32, bitcast=True))
        tl.store(o1 + i, r1.to(tl.int32, bitcast=True))
        tl.store(o2 + i, r2.to(tl.int32, bitcast=True))
        tl.store(o3 + i, r3.to(tl.int32, bitcast=True))

    n = len(c0)
    ins = [torch.tensor(np.asarray(v, dtype=np.uint32).view(np.int32)) for v in (c0, c1, c2, c3)]
    outs = [torch.zeros(n, dtype=torch.int32) for _ in range(4)]
    kern[(1,)](*outs, *ins, seed, N=n)
    return np.stack([o.numpy().view(np.uint32) for o in outs], axis=1)


@pytest.mark.parametrize("seed", [0, 1, 7, 0x5EED0502039, 2**64 - 1, 0x123456789ABCDEF])
def test_philox_matches_triton(seed):
    rng = np.random.default_rng(seed % 1000)
    n = 64
    c0 = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    c1 = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    c2 = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    c3 = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    c0[:4] = [0, 1, 2**32 - 1, 12345]
    c1[:4] = [0, 0, 2**32 - 1, 1]
    c2[:4] = [0, 1, 2**32 - 1, 0]
    c3[:4] = [0, 0, 2**32 - 1, 0]
    ref = _triton_philox(seed, c0, c1, c2, c3)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    got = np.stack([oracle.philox4x32_10([c0[i], c1[i], c2[i], c3[i]], key) for i in range(n)])
    assert np.array_equal(got, ref)


def test_event_and_init_blocks_match_triton():
    """B(c,k) = Philox({c,k,0,0}) and I(c) = Philox({c,0,1,0}) under key (seed lo, seed hi)."""
    seed = 0xDEADBEEF12345
    cells = np.arange(0, 256, dtype=np.uint32) * 7919
    ks = (np.arange(256, dtype=np.uint32) * 13) % 50
    ev = oracle.philox_blocks(seed, cells, ks, 0)
    z = np.zeros_like(cells)
    assert np.array_equal(ev, _triton_philox(seed, cells, ks, z, z))
    ini = oracle.philox_blocks(seed, cells, 0, 1)
    assert np.array_equal(ini, _triton_philox(seed, cells, z, z + 1, z))

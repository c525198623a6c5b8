"""The device integer logarithm equals the oracle's on every one of the 2^32 input words.

exp_ticks (the -ln r of Eq. (5) in integer ticks) is computed on the device in chunks of
2^26 words and compared with the oracle's plain loop, chunk by chunk, through a position-
dependent digest (sums of the 32-bit halves of out ^ (i * 0x9E3779B97F4A7C15), which a
wrong, missing or misplaced word changes); a digest mismatch is then located word by
word.  The oracle side runs in a spawn process pool on the host cores, started before
the first GPU call."""
import multiprocessing as mp
import os

import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CHUNK = 1 << 26
NCHUNK = (1 << 32) // CHUNK
MIX = np.uint64(0x9E3779B97F4A7C15)


def _digest_np(out: np.ndarray, start: int):
    pos = (np.arange(start, start + out.size, dtype=np.uint64) * MIX)
    v = out ^ pos
    lo = (v & np.uint64(0xFFFFFFFF)).astype(np.int64).sum()
    hi = (v >> np.uint64(32)).astype(np.int64).sum()
    return int(lo), int(hi)


def _oracle_chunk(k: int):
    import oracle
    start = k * CHUNK
    x = np.arange(start, start + CHUNK, dtype=np.uint64).astype(np.uint32)
    return k, _digest_np(oracle.exp_ticks_many(x), start)


def test_exp_ticks_all_words():
    ctx = mp.get_context("spawn")
    workers = max(1, min(32, (os.cpu_count() or 2)))
    with ctx.Pool(workers) as pool:
        pending = pool.imap_unordered(_oracle_chunk, range(NCHUNK))
        ac = pytest.importorskip("paper_cs_0502039_gb300")
        torch = pytest.importorskip("torch")
        if not torch.cuda.is_available():
            pytest.skip("no CUDA device")
        mix = torch.tensor(int(MIX) - (1 << 64), dtype=torch.int64, device="cuda")
        dx = torch.empty(CHUNK, dtype=torch.int32, device="cuda")
        dout = torch.empty(CHUNK, dtype=torch.int64, device="cuda")
        base = torch.arange(CHUNK, dtype=torch.int64, device="cuda")
        dev = {}
        for k in range(NCHUNK):
            start = k * CHUNK
            dx.copy_((base + start).to(torch.int64).bitwise_and(0xFFFFFFFF).to(torch.int32))
            ac.ac_dev_exp_ticks(dx.data_ptr(), dout.data_ptr(), CHUNK)
            v = dout ^ ((base + start) * mix)
            lo = (v & 0xFFFFFFFF).sum().item()
            hi = ((v >> 32) & 0xFFFFFFFF).sum().item()
            dev[k] = (int(lo), int(hi))
        bad = []
        for k, dig in pending:
            if dig != dev[k]:
                bad.append(k)
    if bad:
        import oracle
        k = bad[0]
        x = np.arange(k * CHUNK, (k + 1) * CHUNK, dtype=np.uint64).astype(np.uint32)
        dx.copy_(torch.from_numpy(x.view(np.int32)).cuda())
        ac.ac_dev_exp_ticks(dx.data_ptr(), dout.data_ptr(), CHUNK)
        got = dout.cpu().numpy().view(np.uint64)
        want = oracle.exp_ticks_many(x)
        first = int(np.flatnonzero(got != want)[0])
        pytest.fail(f"{len(bad)} chunks differ; first word {x[first]:#x}: device {got[first]}, oracle {want[first]}")

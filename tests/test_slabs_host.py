"""Row slabs, host side (no GPU): the split of the torus rows and the halo exchange over
torch.distributed with the gloo backend, 2 and 3 ranks, on tagged CPU rows."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_cs_0502039_gb300 import slabs


def test_plan_covers_the_torus_once():
    for rows, n, R in [(300, 2, 4), (97, 3, 6), (4096, 8, 8), (64, 4, 4)]:
        p = slabs.plan(rows, n, R)
        covered = np.zeros(rows, int)
        for sl in p:
            covered[sl.row0:sl.row0 + sl.nrows] += 1
            assert R <= sl.nrows <= rows - 2 * R
            assert p[sl.above].row0 + p[sl.above].nrows == sl.row0 or (sl.index == 0 and sl.above == n - 1)
        assert (covered == 1).all()
    with pytest.raises(ValueError):
        slabs.plan(20, 4, 8)          # slabs thinner than the halo
    with pytest.raises(ValueError):
        slabs.plan(20, 1, 8)          # one slab would reach into its own halo


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


ROWS, COLS, R = 30, 5, 3


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    plan = slabs.plan(ROWS, world, R)
    sl = plan[rank]
    # a rank's state: its own rows hold rank-tagged cell values, every other row -1
    state = torch.full((ROWS, COLS * slabs.BYTES_PER_CELL // 4), -1, dtype=torch.int32)
    for r in range(sl.row0, sl.row0 + sl.nrows):
        state[r] = torch.arange(state.shape[1], dtype=torch.int32) + 1000 * r + 100000 * rank
    nbytes = R * COLS * slabs.BYTES_PER_CELL

    def rows_of(row):
        return [(row + k) % ROWS for k in range(R)]

    def export_rows(row, buf):
        buf.view(torch.int32).view(R, -1).copy_(state[rows_of(row)])

    def import_rows(row, buf):
        state[rows_of(row)] = buf.view(torch.int32).view(R, -1)

    slabs.exchange_distributed(export_rows, import_rows, sl, R, nbytes, torch.device("cpu"), dist)
    out[rank] = state.numpy().copy()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_halo_exchange_over_gloo(world):
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    plan = slabs.plan(ROWS, world, R)
    owner = {}
    for sl in plan:
        for r in range(sl.row0, sl.row0 + sl.nrows):
            owner[r] = sl.index
    width = COLS * slabs.BYTES_PER_CELL // 4
    for sl in plan:
        st = out[sl.index]
        above, below = slabs.halo_rows(sl, ROWS, R)
        for r in [(above + k) % ROWS for k in range(R)] + [(below + k) % ROWS for k in range(R)]:
            want = np.arange(width) + 1000 * r + 100000 * owner[r]
            assert np.array_equal(st[r], want), (sl.index, r)

"""Multi-process host logic on CPU (gloo, world size 2): round-robin sharding covers every
lattice once, replica seeds differ per rank, and the end-of-run reduction takes the
maximum time and the total work over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_cs_0502039_gb300 import dist as acdist  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = acdist.rank_env()
    mine = acdist.shard(range(11), r, w)
    t, work = acdist.reduce_run(elapsed_s=1.0 + r, work=len(mine))
    got = [None] * world
    dist.all_gather_object(got, mine)
    out[rank] = (r, w, lr, acdist.replica_seed(7, r), t, work, sorted(x for g in got for x in g))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    assert (r0[0], r0[1], r1[0], r1[1]) == (0, 2, 1, 2)
    assert r0[3] != r1[3]                               # replica seeds differ
    assert r0[4] == r1[4] == 2.0                        # max over ranks
    assert r0[5] == r1[5] == 11                         # total work
    assert r0[6] == list(range(11))                     # every lattice exactly once


def test_replica_seeds_are_injective():
    seen = {acdist.replica_seed(seed, rank) for seed in (0, 1, 999, 1000, 1001, (1 << 48) - 1) for rank in range(8)}
    assert len(seen) == 6 * 8
    assert acdist.replica_seed(7, 0) == 7
    with pytest.raises(ValueError):
        acdist.replica_seed(1 << 48, 0)


def test_single_process_identity():
    assert acdist.reduce_run(3.5, 10) == (3.5, 10.0)
    assert acdist.shard([1, 2, 3], 0, 1) == [1, 2, 3]

"""The N-rank bench path on CPU (gloo, world size 2): ranks decode disjoint seeded
batches and only the job time is reduced (max over ranks)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    got = bench.max_over_ranks(10.0 + rank)
    code, llr = bench.make_workload(3, rank)
    out[rank] = (got, float(np.abs(llr).sum()), tuple(bench.workload_seeds(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 11.0  # every rank reports the slowest rank's time
    assert res[0][2] != res[1][2] and not set(res[0][2]) & set(res[1][2])  # disjoint seeds
    assert res[0][1] != res[1][1]  # different frames


def test_single_process_max_is_identity():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5

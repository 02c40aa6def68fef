"""The N > 1 path of bench.py on the host: one process per rank (here two
gloo ranks on the CPU), the job time is the slowest rank's, and every rank
runs its own replica of the workload (no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as tdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist()
    t = bench.max_over_ranks(1.5 + rank)          # rank 1 is the slow one
    tdist.barrier()
    out[rank] = (ws, r, local, t)
    tdist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    assert res[0] == (2, 0, 0, 2.5) and res[1] == (2, 1, 1, 2.5)


def test_single_process_is_its_own_maximum():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25

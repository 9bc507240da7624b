"""The replicas path of bench.py (N > 1): whole-job value = edges of all ranks
over the slowest rank's time, computed with a collective -- two gloo ranks on
the CPU."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [100.0, 140.0][rank]
    edges = [1e9, 3e9][rank]
    t, e = bench.aggregate_ranks(ms, edges, world, "cpu")
    out[rank] = (t, e)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        t, e = out[r]
        assert t == 140.0 and e == 4e9          # max time, summed edges
    assert abs(out[0][1] / (out[0][0] / 1e3) - 4e9 / 0.14) < 1


def test_single_rank_is_identity():
    import bench
    assert bench.aggregate_ranks(5.0, 7.0, 1) == (5.0, 7.0)

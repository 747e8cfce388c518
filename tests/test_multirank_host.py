"""N > 1 path of bench.py on CPU: two gloo ranks with independent results; the
combined figures are the slowest rank's time and the sum of the nodes."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, nodes = bench.combine_ranks(100.0 + 50.0 * rank, 1000 + rank, world)
    out[rank] = (ms, nodes)
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_gloo_world2():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (150.0, 2001.0)

"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank
draws its own batch of maps (weak scaling, no data exchange) and the job time
is the maximum over ranks."""
import os
import socket

import numpy as np


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    c, maps = bench.workload(rank)
    fingerprint = [complex(f[5]) for f, _, _ in maps]
    m = bench.reduce_max(10.0 * (rank + 1), dist)
    q.put((rank, fingerprint, m, [len(p) for _, _, p in maps]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_disjoint_batches_and_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (r0, fp0, m0, n0), (r1, fp1, m1, n1) = out
    assert m0 == m1 == 20.0
    assert n0 == n1 == [930, 930, 930, 930]
    assert not np.allclose(fp0, fp1)            # different seeds: no rank repeats another's maps
    assert len(set(fp0 + fp1)) == 8

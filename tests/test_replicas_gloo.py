"""The multi-GPU replica path on CPU: two gloo ranks, distinct seeds, max-over-ranks timing."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    from paper_1709_06350_gb300 import replicas, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, lr = replicas.world()
    seed = replicas.replica_seed(3000, r)
    d, _ = synth.linear_field(16, 16.0, 1.0, seed)
    replicas.barrier(dist)
    elapsed = 1.0 + r                       # rank 1 is the slow one
    worst = replicas.max_over_ranks(elapsed, dist)
    out[rank] = (ws, r, seed, float(d[0, 0, 0]), worst,
                 replicas.job_throughput(2.0, ws, worst))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    a, b = out[0], out[1]
    assert (a[0], a[1], b[1]) == (2, 0, 1)
    assert a[2] == 3000 and b[2] != a[2] and a[3] != b[3]     # independent realisations
    assert a[4] == b[4] == 2.0                               # max over ranks
    assert a[5] == pytest.approx(2.0)                        # 2 units x 2 ranks / 2 s

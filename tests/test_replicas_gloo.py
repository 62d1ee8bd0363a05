"""Multi-process host logic of replica runs on CPU with gloo (world size 2):
the whole-job rate uses every rank's units over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2312_10070_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        replicas.barrier()
        local_s = [2.0, 3.0][rank]        # rank 1 is the slower replica
        rate = replicas.whole_job_rate(100.0, local_s)
        mx = replicas.max_over_ranks(float(rank + 10))
        out.put((rank, replicas.world(), rate, mx))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, rate, mx in res:
        assert w == 2
        assert rate == pytest.approx(2 * 100.0 / 3.0)
        assert mx == 11.0


def test_single_process_defaults():
    from paper_2312_10070_gb300 import replicas
    assert replicas.world() == 1
    assert replicas.max_over_ranks(4.5) == 4.5
    assert replicas.whole_job_rate(10.0, 2.0) == 5.0

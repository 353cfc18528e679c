"""The multi-rank reductions of the benchmark on CPU (gloo, world size 2):
max-over-ranks time and whole-job rate, replicas only."""
import os
import socket

import torch.multiprocessing as mp

from paper_1305_2418_gb300 import dist as D


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = D.env()
    # rank r "processed" 100*(r+1) units in (10 + 5 r) ms
    rate, ms = D.whole_job_rate(100.0 * (r + 1), 10.0 + 5.0 * r)
    dist.barrier()
    q.put((r, w, lr, rate, ms))
    dist.destroy_process_group()


def test_whole_job_rate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, w, lr, rate, ms) in enumerate(res):
        assert (rank, w, lr) == (r, 2, r)
        assert ms == 15.0                       # max over ranks
        assert abs(rate - 300.0 / 0.015) < 1e-6  # all units / slowest rank


def test_single_process_is_identity():
    rate, ms = D.whole_job_rate(50.0, 20.0)
    assert ms == 20.0 and abs(rate - 2500.0) < 1e-9
